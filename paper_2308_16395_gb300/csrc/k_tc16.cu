// FP16-split tensor-core pass of a spatial mode (Alg. 4: projection P_k, residual E_k and its
// norm), with the input tile held in tensor memory so that the residual needs no second read of
// the input.
//
// The mode-k input X (row-major F x n_k, the mode-k fibers as rows) streams through shared memory
// by TMA in chunks of 128 fibers x 64 columns (two 32-column boxes, 128-byte swizzle). Eight
// splitter warps convert each chunk in place into the FP16 high and low parts of X_s = 2^sigma X
// (x_s = hi + lo up to 2^-23 |x_s| + 2^-25) for MMA1 and, in the residual passes, then store the
// FP32 values X_s into tensor memory (lane = fiber, one column per element).
//   MMA1  P_s = X_s (2^14 U_k) on kind::f16, three products per K step of 16 (hi*hi into one
//         accumulator, hi*lo + lo*hi into a second; FP16 products are exact in FP32), U_k's FP16
//         parts streamed with the chunks.
//   epi-1 P = 2^-(sigma+14) P_s into a shared staging tile; -2^-19 P_s split into FP16 hi/lo in
//         tensor memory over the accumulators just read (MMA2's A operand).
//   MMA2  accumulated onto the stored tile: X_s + (-2^-19 P_s)(2^5 U_k)^T = 2^sigma (X - P U_k^T)
//         = 2^sigma E, three products per K step, in 128-column blocks; each block's FP16 parts
//         of 2^5 U_k (128 rows) come round the input ring after the tile's chunks, so that the
//         ring has four stages (more input in flight) instead of two beside resident rows.
//   epi-2 ||E||^2 per CTA (FP32 over 32 columns of a fiber, then FP64), E^T for the residual
//         Gram when the mode grew.
//   out   two otherwise idle warps write the staged P to global memory, column-major (F x r_k,
//         the next mode's input), while the epilogue goes on to E.
// epi-2 is the splitters' own: before a splitter warp stores its 32 columns of a chunk it reads
// the previous tile's E at those columns (once MMA2 has completed their 128-column block), so a
// column is overwritten only by the thread that read it and no hand-over is needed; the
// splitters hand each chunk's FP16 parts to MMA1 before that read, so the next tile's MMA1
// follows MMA2 on the tensor pipe without waiting for it. The ring of input stages is fed from
// L2, into which the producer prefetches chunks ahead.
//
// Scale: sigma_k (Ctl::x16e) puts the input's largest |x| near 2^8, far from the FP16 limits
// (|x_s| <= 2^15 keeps hi finite; the low end loses only an absolute 2^-25). Pass A records
// max |x| (Ctl::xmax); a second launch of pass A right after it returns at once unless the scaled
// maximum left [2^1, 2^15), and then runs the pass again with sigma from that maximum. With
// |x_s| < 2^15, |U| <= 1 and |p| <= sqrt(n_k) max|x| (orthonormal U_k), every FP16 operand
// stays below 2^15 for n_k <= 384 (|2^-19 P_s| <= 2^-5 sqrt(n_k) max|x_s|).
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"
#include "tc_common.cuh"

namespace tk {

using namespace tc;

constexpr int H_M = 128;                         // fibers per tile
constexpr int H_KC = 64;                         // input columns per chunk
constexpr int H_XB = H_M * H_KC * 4;             // 32 KB: raw FP32 chunk, then FP16 hi | lo
constexpr int H_UB = TP_RMAX * 128;              // 8 KB: U chunk (hi or lo), <= 64 rows x 128 B
constexpr int H_STAGE = H_XB + 2 * H_UB;         // 48 KB
constexpr int H_PST = TP_RMAX * H_M * 4;         // 32 KB: staged P tile, [column][fiber] FP32
constexpr int H_PF = 6;                          // chunks prefetched into L2 ahead of the loads
constexpr int H_SPLIT_W = 8;                     // splitter warps 4..11
constexpr int H_EPI_W0 = 12;                     // epilogue warps 12..15
constexpr int H_NT = 32 * 16;
constexpr int H_TP = TK_H16_NMAX;                // TMEM column of the P accumulators
constexpr uint32_t H_TMEM_COLS = 512;
static_assert(H_TP + 2 * TP_RMAX <= (int)H_TMEM_COLS, "input tile and P accumulators fit TMEM");
// MMA2's A operand over the accumulators: K columns 0..31 (packed two per TMEM column) of the
// high part at H_TP, of the low part at H_TP + 16 (both over P columns 0..31 of the hi*hi
// accumulator, read first); K columns 32..63 at H_TP + 64 and H_TP + 80 (over P columns 0..31
// of the correction accumulator, also read first)
__device__ __forceinline__ uint32_t a16_col(int ks, int lo) {
  return (uint32_t)(H_TP + (ks < 2 ? 0 : TP_RMAX) + 16 * lo + 8 * (ks & 1));
}

// Four stages in both forms; in the residual form MMA2's U_k rows go round the same ring (one
// item per 128-row block after a tile's input chunks) instead of staying resident.
template <bool RESID> struct HCfg {
  static constexpr int S = 4;
  static constexpr size_t EXTRA = H_PST;
  static constexpr size_t SMEM = (size_t)S * H_STAGE + EXTRA + 1024 + 1024;
};
static_assert(H_XB / 2 >= 128 * 128, "a stage holds a 128-row block of U_k's FP16 hi and lo rows");
static_assert(HCfg<true>::SMEM <= 232448, "shared memory of the residual pass");
static_assert(HCfg<false>::SMEM <= 232448, "shared memory of the projection pass");

// Bounded wait (1 s of wall time); sets *abort on timeout, returns false once aborted.
__device__ __forceinline__ unsigned long long h_timer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool h_wait(uint64_t* bar, uint32_t parity, volatile int* abort) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = h_timer();
  for (long long i = 0;; ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 63) {
      if (*abort) return false;
      if (h_timer() - t0 > 1000000000ull) { *abort = 1; return false; }
    }
  }
}
// Wait (0.2 s at most, whatever *abort says) for copies or MMAs this CTA has in flight, before
// its shared and tensor memory go away.
__device__ __forceinline__ void h_drain(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return;
  const unsigned long long t0 = h_timer();
  while (!mbar_try_wait(bar, parity))
    if (h_timer() - t0 > 200000000ull) return;
}

__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
  return *reinterpret_cast<uint32_t*>(&h);
}

// FP16 hi/lo of a pair: a = hi + lo up to the rounding of lo.
__device__ __forceinline__ void split_h2(float a0, float a1, uint32_t& hi, uint32_t& lo) {
  const __half2 h = __floats2half2_rn(a0, a1);
  const float2 hf = __half22float2(h);
  hi = h2_bits(h);
  lo = h2_bits(__floats2half2_rn(a0 - hf.x, a1 - hf.y));
}

struct TcPass16Args {
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
  int rerun;                // the second launch of pass A (runs only outside the scale window)
  int track;                // record max |x| (pass A)
};

template <bool RESID, bool WRITE_ET>
__global__ void __launch_bounds__(H_NT, 1) k_tc_pass16(Ctl* __restrict__ ctl, int pred,
                                                     const __grid_constant__ CUtensorMap mY,
                                                     const __grid_constant__ CUtensorMap mD0,
                                                     const __grid_constant__ CUtensorMap mD1,
                                                     const __grid_constant__ CUtensorMap mD2,
                                                     const __grid_constant__ CUtensorMap mU1hi,
                                                     const __grid_constant__ CUtensorMap mU1lo,
                                                     const __grid_constant__ CUtensorMap mU2hi,
                                                     const __grid_constant__ CUtensorMap mU2lo,
                                                     TcPass16Args a) {
  if (ctl->status) return;
  const int k = a.k;
  if (pred && !ctl->grew[k]) return;
  const int r = ctl->r[k];
  if (!tc_proj_ok(ctl, k, r)) return;
  const int n1 = ctl->n[k];
  if (n1 > TK_H16_NMAX) return;
  int sigma = ctl->x16e[k];
  if (a.rerun) {
    const unsigned mb = ctl->xmax[k];
    if (mb == 0u || mb >= 0x7f800000u) return;
    const int em = x16_exp_of_bits(mb);
    if (x16_in_window(em, sigma)) return;
    sigma = x16_sigma_for(em);
  }
  const long long F = view_B(ctl, k);
  const int Rp = (r + 15) / 16 * 16;
  const int n1p = (n1 + 15) / 16 * 16;
  const int Kc = (n1 + H_KC - 1) / H_KC;
  const int nblk = (n1p + 127) / 128;
  const long long ntiles = (F + H_M - 1) / H_M;
  const int xb = ctl->xbuf;
  const CUtensorMap* mX = xb < 0 ? (a.mYg ? a.mYg : &mY) : (xb == 0 ? &mD0 : (xb == 1 ? &mD1 : &mD2));
  float* P = a.dbufs[(xb + a.out_off + 3) % 3];

  extern __shared__ __align__(1024) unsigned char hsm_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(hsm_raw) + 1023) & ~uintptr_t(1023));
  constexpr int S = HCfg<RESID>::S;
  float* Pst = reinterpret_cast<float*>(base + (size_t)S * H_STAGE);
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + (size_t)S * H_STAGE + HCfg<RESID>::EXTRA);
  uint64_t* full = bars;                 // [S] chunk landed
  uint64_t* conv = bars + S;             // [S] chunk's FP16 parts in shared memory
  uint64_t* empty = bars + 2 * S;        // [S] chunk's MMAs done
  uint64_t* d1full = bars + 3 * S;       // P accumulators complete
  uint64_t* pready = d1full + 1;         // P read out (MMA2's A operand stored over it)
  uint64_t* efull = pready + 1;          // [3] E block b complete
  uint64_t* xst = efull + 3;             // the tile's input stored in tensor memory
  uint64_t* done = xst + 1;              // every MMA complete
  uint64_t* pstaged = done + 1;          // the tile's P in the staging tile
  uint64_t* pfree = pstaged + 1;         // the staging tile written out
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(pfree + 1);
  volatile int* abort = reinterpret_cast<volatile int*>(tmem_slot + 1);
  double* red = reinterpret_cast<double*>(tmem_slot + 4);        // [16] per-warp sums
  unsigned* redm = reinterpret_cast<unsigned*>(red + 16);        // [16] per-warp max |x|
  double* rede = reinterpret_cast<double*>(redm + 16);           // [16] per-warp ||E||^2

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 32 * H_SPLIT_W);
      mbar_init(&empty[s], 1);
    }
    mbar_init(d1full, 1);
    mbar_init(pready, 128);
    for (int b = 0; b < 3; ++b) {
      mbar_init(&efull[b], 1);
    }
    mbar_init(xst, 32 * H_SPLIT_W);
    mbar_init(done, 1);
    mbar_init(pstaged, 128);
    mbar_init(pfree, 64);
    *abort = 0;
    fence_barrier_init();
  }
  if (threadIdx.x < 16) {
    red[threadIdx.x] = 0.0;
    redm[threadIdx.x] = 0u;
    rede[threadIdx.x] = 0.0;
  }
  if (warp == 1) {
    tmem_alloc(tmem_slot, H_TMEM_COLS);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const long long myt = ntiles > blockIdx.x ? (ntiles - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;

  // test hook: the producer issues nothing, so the consumers' waits run out (1 s), the CTA
  // latches TUCKER_ETIMEOUT and ends normally
  const bool stall = a.track && k == 0 && ctl->test_stall != 0;
  if (warp == 0) {
    if (lane == 0 && !stall) {
      // ---------------- TMA producer ----------------
      if (xb < 0 && a.mYg) tensormap_acquire(a.mYg);
      tma_prefetch(mX);
      tma_prefetch(&mU1hi);
      tma_prefetch(&mU1lo);
      const int u2rows = (n1p + 63) / 64 * 64;
      if (RESID) {
        tma_prefetch(&mU2hi);
        tma_prefetch(&mU2lo);
      }
      const long long nq = myt * Kc;
      auto prefetch_chunk = [&](long long qq) {
        if (qq >= nq) return;
        const long long tt = blockIdx.x + (qq / Kc) * (long long)gridDim.x;
        const int x0 = (int)(qq % Kc) * H_KC;
        tma_prefetch_l2_2d(mX, x0, (int)(tt * H_M));
        if (x0 + 32 < n1) tma_prefetch_l2_2d(mX, x0 + 32, (int)(tt * H_M));
      };
      for (long long qq = 0; qq < H_PF; ++qq) prefetch_chunk(qq);
      long long q = 0, qx = 0;   // ring items; input chunks among them
      bool ok = true;
      for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x) {
        for (int c = 0; c < Kc; ++c, ++q, ++qx) {
          const int s = (int)(q % S);
          prefetch_chunk(qx + H_PF);
          if (!h_wait(&empty[s], (uint32_t)(((q / S) & 1) ^ 1), abort)) { ok = false; break; }
          unsigned char* st = base + (size_t)s * H_STAGE;
          mbar_arrive_expect_tx(&full[s], (uint32_t)(H_XB + Rp * 128 * 2));
          // the second box may lie wholly past n_k: TMA writes zeros there
          tma_load_2d(mX, &full[s], st, c * H_KC, (int)(t * H_M));
          tma_load_2d(mX, &full[s], st + H_XB / 2, c * H_KC + 32, (int)(t * H_M));
          for (int n0 = 0; n0 < Rp; n0 += 16) {
            tma_load_2d(&mU1hi, &full[s], st + H_XB + n0 * 128, c * H_KC, n0);
            tma_load_2d(&mU1lo, &full[s], st + H_XB + H_UB + n0 * 128, c * H_KC, n0);
          }
        }
        if (!RESID || !ok) continue;
        // MMA2's U_k rows, one 128-row block per item (FP16 hi, then lo 16 KB further); rows past
        // n_k arrive as zeros
        for (int b = 0; b < nblk; ++b, ++q) {
          const int s = (int)(q % S);
          if (!h_wait(&empty[s], (uint32_t)(((q / S) & 1) ^ 1), abort)) { ok = false; break; }
          unsigned char* st = base + (size_t)s * H_STAGE;
          const int r1 = min(128 * b + 128, u2rows);
          mbar_arrive_expect_tx(&full[s], (uint32_t)(r1 - 128 * b) * 128u * 2u);
          for (int r0 = 128 * b; r0 < r1; r0 += 64) {
            tma_load_2d(&mU2hi, &full[s], st + (size_t)(r0 - 128 * b) * 128, 0, r0);
            tma_load_2d(&mU2lo, &full[s], st + H_XB / 2 + (size_t)(r0 - 128 * b) * 128, 0, r0);
          }
        }
      }
      // every load issued has landed before the CTA's shared memory goes away
      for (long long j = (q > S ? q - S : 0); j < q; ++j) h_drain(&full[j % S], (uint32_t)((j / S) & 1));
    }
    __syncwarp();
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t id1 = idesc_f16(H_M, Rp);
      const uint32_t tP = tmem + H_TP, tC = tmem + H_TP + TP_RMAX;
      bool ok = true;
      long long q = 0;
      uint32_t cpar = 0u;   // bit s: parity of stage s's next input-chunk conversion
      int it = 0;
      for (long long t = blockIdx.x; ok && t < ntiles; t += gridDim.x, ++it) {
        // projection form: the P accumulators are free once the epilogue has read the previous
        // tile's (in the residual form MMA2 of the previous tile, issued before, waited for that)
        if (!RESID && it > 0 && !h_wait(pready, (uint32_t)((it - 1) & 1), abort)) { ok = false; break; }
        tc_fence_after();
        for (int c = 0; c < Kc; ++c, ++q) {
          const int s = (int)(q % S);
          if (!h_wait(&conv[s], (cpar >> s) & 1u, abort)) { ok = false; break; }
          cpar ^= 1u << s;
          tc_fence_after();
          unsigned char* st = base + (size_t)s * H_STAGE;
          const uint64_t ahi = desc_sw128(st), alo = desc_sw128(st + H_XB / 2);
          const uint64_t bhi = desc_sw128(st + H_XB), blo = desc_sw128(st + H_XB + H_UB);
#pragma unroll
          for (int k4 = 0; k4 < H_KC / 16; ++k4) {
            const uint64_t o = (uint64_t)(k4 * 32) >> 4;
            const uint32_t acc = (c | k4) ? 1u : 0u;
            mma_f16(tP, ahi + o, bhi + o, id1, acc);
            mma_f16(tC, ahi + o, blo + o, id1, acc);
            mma_f16(tC, alo + o, bhi + o, id1, 1u);
          }
          tc_commit(&empty[s]);
        }
        if (!ok) break;
        tc_commit(d1full);
        if (RESID) {
          // E = X - P U^T onto the stored tile, once P's FP16 parts are in tensor memory and the
          // tile's input is stored
          if (!h_wait(pready, (uint32_t)(it & 1), abort)) { ok = false; break; }
          if (!h_wait(xst, (uint32_t)(it & 1), abort)) { ok = false; break; }
          tc_fence_after();
          for (int b = 0; b < nblk; ++b, ++q) {
            // block b of U_k's rows landed in its ring stage
            const int s = (int)(q % S);
            if (!h_wait(&full[s], (uint32_t)((q / S) & 1), abort)) { ok = false; break; }
            tc_fence_after();
            unsigned char* st = base + (size_t)s * H_STAGE;
            const int c0 = 128 * b;
            const int nc = min(128, n1p - c0);
            const uint32_t idb = idesc_f16(H_M, nc);
            const uint64_t uhi = desc_sw128(st), ulo = desc_sw128(st + H_XB / 2);
            for (int ks = 0; ks < Rp / 16; ++ks) {
              const uint64_t o = (uint64_t)(ks * 32) >> 4;
              mma_f16_ts(tmem + c0, tmem + a16_col(ks, 0), uhi + o, idb, 1u);
              mma_f16_ts(tmem + c0, tmem + a16_col(ks, 0), ulo + o, idb, 1u);
              mma_f16_ts(tmem + c0, tmem + a16_col(ks, 1), uhi + o, idb, 1u);
            }
            tc_commit(&efull[b]);
            tc_commit(&empty[s]);
          }
          if (!ok) break;
        }
      }
      tc_commit(done);
      h_drain(done, 0);
    }
    __syncwarp();
  } else if (warp == 2 || warp == 3) {
    // ---------------- P writers: the staged P out (passes that write P) ----------------
    if (!WRITE_ET) {
      int it = 0;
      for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
        const bool okw = h_wait(pstaged, (uint32_t)(it & 1), abort);
        if (bar_any(3, 64, !okw)) break;
        // column-major (F x r): a warp writes 32 consecutive fibers of a column at a time
        const long long f0 = t * H_M;
        for (int c = warp - 2; c < r; c += 2) {
          const float* src = Pst + c * H_M;
          float* dst = P + F * c + f0;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (f0 + 32 * j + lane < F) dst[32 * j + lane] = src[32 * j + lane];
        }
        // the staging tile is free again for the next tile's epi-1
        mbar_arrive(pfree);
      }
    }
  } else if (warp >= 4 && warp < 4 + H_SPLIT_W) {
    // ---------------- splitters ----------------
    const int q4 = warp & 3, h = (warp - 4) >> 2;
    const int row = q4 * 32 + lane;
    const uint32_t lq = (uint32_t)(q4 * 32) << 16;
    const float sc = pow2f(sigma), eun = pow2f(-sigma);
    float xm = 0.f;
    double yacc = 0.0, eacc = 0.0;
    long long q = 0;
    int it = 0;
    bool stop = false, okx = true;
    // epi-2 at this warp's 32 tensor-memory columns cb .. cb + 31 of the tile whose lane-`row`
    // fiber is f: ||E||^2 (FP32 over the 32 columns, then FP64) and E^T when the mode grew
    auto e_cols = [&](int cb, long long f) {
      uint32_t e[32];
      tmem_ld32_nw(tmem + lq + (uint32_t)cb, e);
      tmem_ld_wait();
      const bool live = f < F;
      float eb = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const float ev = __uint_as_float(e[i]) * eun;
        if (cb + i < n1) {
          eb = fmaf(ev, ev, eb);
          if (WRITE_ET) {
            if (live) a.Et[(long long)(cb + i) * a.et_stride + f] = ev;
            else if (f < a.et_stride) a.Et[(long long)(cb + i) * a.et_stride + f] = 0.f;
          }
        }
      }
      if (live) eacc += (double)eb;
    };
    for (long long t = blockIdx.x; !stop && t < ntiles; t += gridDim.x, ++it) {
      float yt = 0.f;   // FP32 over the tile's chunks (<= 6 sums of 32 terms), FP64 per tile
      const long long fprev = (t - gridDim.x) * H_M + row;   // this lane's fiber, tile before
      for (int c = 0; c < Kc; ++c, ++q) {
        const int s = (int)(q % S);
        const bool ok = h_wait(&full[s], (uint32_t)((q / S) & 1), abort);
        unsigned char* st = base + (size_t)s * H_STAGE;
        float x[32];
        const float4* src = reinterpret_cast<const float4*>(st + h * (H_XB / 2) + row * 128);
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const float4 v = src[u ^ (row & 7)];
          x[4 * u] = v.x; x[4 * u + 1] = v.y; x[4 * u + 2] = v.z; x[4 * u + 3] = v.w;
        }
        // every splitter has read the stage before any writes its FP16 parts over it (and a
        // wait that gave up, here or on the previous chunk's block, stops all of them)
        if (bar_any(1, 32 * H_SPLIT_W, !(ok && okx))) { stop = true; break; }
        float ys = 0.f;
        uint32_t hp[16], lp[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const float a0 = x[2 * i], a1 = x[2 * i + 1];
          ys = fmaf(a0, a0, ys);
          ys = fmaf(a1, a1, ys);
          xm = fmaxf(xm, fmaxf(fabsf(a0), fabsf(a1)));
          x[2 * i] = a0 * sc;
          x[2 * i + 1] = a1 * sc;
          split_h2(x[2 * i], x[2 * i + 1], hp[i], lp[i]);
        }
        yt += ys;
        // hi row `row`: FP16 columns 32 h .. 32 h + 31 are 16-byte pieces 4 h .. 4 h + 3
        uint4* dh = reinterpret_cast<uint4*>(st + row * 128);
        uint4* dl = reinterpret_cast<uint4*>(st + H_XB / 2 + row * 128);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int u = (4 * h + j) ^ (row & 7);
          dh[u] = make_uint4(hp[4 * j], hp[4 * j + 1], hp[4 * j + 2], hp[4 * j + 3]);
          dl[u] = make_uint4(lp[4 * j], lp[4 * j + 1], lp[4 * j + 2], lp[4 * j + 3]);
        }
        fence_proxy_async_smem();
        mbar_arrive(&conv[s]);
        if (RESID) {
          // this warp's columns of the chunk: first the previous tile's E there (once MMA2 has
          // completed its 128-column block), then the chunk's FP32 values over it; a column is
          // overwritten only by the thread that read it
          const int cb = c * H_KC + 32 * h;
          if (it > 0) {
            okx = h_wait(&efull[c >> 1], (uint32_t)((it - 1) & 1), abort);
            okx = __all_sync(0xffffffffu, okx);
            if (okx) {
              tc_fence_after();
              e_cols(cb, fprev);
            }
          }
          if (okx) {
            tc_fence_after();
            tmem_st32(tmem + lq + (uint32_t)cb, x);
            if (c == Kc - 1) {
              tc_fence_before();
              mbar_arrive(xst);
            }
          }
        }
      }
      yacc += (double)yt;
      if (RESID) q += nblk;   // the tile's U_k-row items, which the MMA issuer takes
    }
    // residual form: E of this CTA's last tile
    if (RESID && !stop && it > 0) {
      const long long flast = (blockIdx.x + (long long)(it - 1) * gridDim.x) * H_M + row;
      for (int c = 0; c < Kc; ++c) {
        const bool oke = h_wait(&efull[c >> 1], (uint32_t)((it - 1) & 1), abort);
        if (bar_any(1, 32 * H_SPLIT_W, !oke)) break;
        tc_fence_after();
        e_cols(c * H_KC + 32 * h, flast);
      }
    }
    const double sy = warp_sum(yacc);
    const double se = warp_sum(eacc);
    float m = xm;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) {
      red[warp] = sy;
      rede[warp] = se;
      redm[warp] = __float_as_uint(m);
    }
  } else if (warp >= H_EPI_W0) {
    // ---------------- epilogue: P (epi-1) into the staging tile ----------------
    const int q4 = warp & 3;
    const int row = q4 * 32 + lane;
    const uint32_t lq = (uint32_t)(q4 * 32) << 16;
    const float pun = pow2f(-(sigma + 14)), pneg = -pow2f(-19);
    constexpr bool OUT = !WRITE_ET;   // this pass writes P
    int it = 0;
    // every give-up below is decided for the four warps together (none of them may leave the
    // loop alone)
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
      bool okw = h_wait(d1full, (uint32_t)(it & 1), abort);
      // the P writers have written the previous tile's P out of the staging tile
      if (OUT && it > 0 && okw) okw = h_wait(pfree, (uint32_t)((it - 1) & 1), abort);
      if (bar_any(2, 128, !okw)) break;
      tc_fence_after();
      // P = sum of the two accumulators, 32 columns at a time
      for (int c0 = 0; c0 < Rp; c0 += 32) {
        float v[32];
        {
          uint32_t a0[32], a1[32];
          tmem_ld32_nw(tmem + lq + H_TP + c0, a0);
          tmem_ld32_nw(tmem + lq + H_TP + TP_RMAX + c0, a1);
          tmem_ld_wait();
#pragma unroll
          for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(a0[i]) + __uint_as_float(a1[i]);
        }
        if (OUT) {
#pragma unroll
          for (int i = 0; i < 32; ++i) Pst[(c0 + i) * H_M + row] = v[i] * pun;
        }
        if (RESID) {
          // MMA2's A operand over accumulator columns read already (see a16_col)
          uint32_t hp[16], lp[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) split_h2(v[2 * i] * pneg, v[2 * i + 1] * pneg, hp[i], lp[i]);
          tmem_st16_nw(tmem + lq + a16_col(c0 >> 4, 0), hp);
          tmem_st16_nw(tmem + lq + a16_col(c0 >> 4, 1), lp);
        }
      }
      if (RESID) tmem_st_wait();
      tc_fence_before();
      mbar_arrive(pready);
      if (OUT) mbar_arrive(pstaged);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) tmem_dealloc(tmem, H_TMEM_COLS);
  if (threadIdx.x == 0) {
    if (*abort) ctl->status = TK_ETIMEOUT;
    double te = 0.0, ty = 0.0;
    unsigned mb = 0u;
    for (int w = 4; w < 4 + H_SPLIT_W; ++w) {
      ty += red[w];
      te += rede[w];
      mb = max(mb, redm[w]);
    }
    if (RESID && !WRITE_ET) {
      for (int j = blockIdx.x; j < a.nparts; j += gridDim.x) {
        a.part_e2[j] = (j == (int)blockIdx.x) ? te : 0.0;
        if (a.part_y2) a.part_y2[j] = (j == (int)blockIdx.x) ? ty : 0.0;
      }
    }
    if (a.track) atomicMax(&ctl->xmax[k], mb);
  }
}

// FP16 hi/lo parts of U_k for the FP16 passes (after the initial ST-HOSVD and after growth):
// U1 = 2^14 U_k as 64 rows x ld1 (row i = column i of U_k, zero past r_k; MMA1's B) and
// U2 = 2^5 U_k as n_k rows x 64 (row j = row j of U_k, zero past r_k; MMA2's B).
__global__ void k_split_u16(const Ctl* ctl, int k, int pred, const double* U, int ldu, int ld1,
                            __half* u1hi, __half* u1lo, __half* u2hi, __half* u2lo) {
  if (ctl->status) return;
  if (pred && !ctl->grew[k]) return;
  const int n1 = ctl->n[k];
  const int r = ctl->r[k];
  for (long long L = blockIdx.x * (long long)blockDim.x + threadIdx.x; L < (long long)TP_RMAX * n1;
       L += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(L % n1), i = (int)(L / n1);
    const float u = (i < r) ? (float)U[(long long)i * ldu + j] : 0.f;
    const float v1 = u * 16384.f, v2 = u * 32.f;
    const __half h1 = __float2half_rn(v1), h2 = __float2half_rn(v2);
    u1hi[(long long)i * ld1 + j] = h1;
    u1lo[(long long)i * ld1 + j] = __float2half_rn(v1 - __half2float(h1));
    u2hi[(long long)j * TP_RMAX + i] = h2;
    u2lo[(long long)j * TP_RMAX + i] = __float2half_rn(v2 - __half2float(h2));
  }
}

cudaError_t launch_split_u16(const Ctl* ctl, int k, int pred, const double* U, int ldu, int ld1,
                             void* const* u16, cudaStream_t st) {
  k_split_u16<<<64, 256, 0, st>>>(ctl, k, pred, U, ldu, ld1, (__half*)u16[0], (__half*)u16[1],
                                  (__half*)u16[2], (__half*)u16[3]);
  return cudaGetLastError();
}

cudaError_t launch_tc_pass16(Ctl* ctl, int k, int mode, int pred, int rerun, const float* Y,
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
  TcPass16Args a{mYg, (float* const*)dbufs, out_off, part_e2, part_y2, nparts, Y, Et, et_stride, k,
                 rerun, mode == 1 ? 1 : 0};
  static bool attr[3] = {false, false, false};
  if (mode == 0) {
    if (!attr[0]) { cudaFuncSetAttribute(k_tc_pass16<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HCfg<false>::SMEM); attr[0] = true; }
    k_tc_pass16<false, false><<<grid, H_NT, HCfg<false>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.h1hi, m.h1lo, m.h2hi, m.h2lo, a);
  } else if (mode == 1) {
    if (!attr[1]) { cudaFuncSetAttribute(k_tc_pass16<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HCfg<true>::SMEM); attr[1] = true; }
    k_tc_pass16<true, false><<<grid, H_NT, HCfg<true>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.h1hi, m.h1lo, m.h2hi, m.h2lo, a);
  } else {
    if (!attr[2]) { cudaFuncSetAttribute(k_tc_pass16<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)HCfg<true>::SMEM); attr[2] = true; }
    k_tc_pass16<true, true><<<grid, H_NT, HCfg<true>::SMEM, st>>>(ctl, pred, mY, m.d[0], m.d[1], m.d[2], m.h1hi, m.h1lo, m.h2hi, m.h2lo, a);
  }
  return cudaGetLastError();
}

}  // namespace tk
