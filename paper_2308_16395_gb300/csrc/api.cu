// C ABI of the streaming ST-HOSVD library: state management and the host-side launch sequence
// of the batch ST-HOSVD (Alg. 2) and of the streaming update (Alg. 5). The update itself is a
// fixed sequence of kernel launches whose data-dependent branches are taken on the device, so
// tucker_stream_update never waits for the device.
#include <stdio.h>
#include <string.h>

#include <stddef.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "../../include/tucker_stream.h"
#include "common.cuh"
#include "kernels.cuh"

using namespace tk;

namespace {

constexpr int kGridP = 152 * 2;    // projection kernel grid (persistent-style, grid-stride)
constexpr int kGridI = 152 * 2;    // ISVD row-pass grid (one wave at two blocks per SM)
constexpr int kGridCV = 152 * 4;   // core / V update grid
constexpr int kGramBlocks = 600;   // target blocks of the residual-Gram kernel
constexpr int kSecMax = TK_STREAM_CAP_MAX + 2;

}  // namespace

struct tucker_state {
  tucker_config cfg{};
  int d = 0;
  int n[TK_MAXD]{};
  int cap[TK_MAXD]{};
  long long core_cap = 0;
  int steps_cap = 0;
  int ldc = 0;
  int tw = 8;          // bytes of the work type
  int tx = 8;          // bytes of the slice type
  long long N = 0;     // elements per slice
  int nmax = 0;        // largest eigenproblem
  int mcap = 0;        // largest number of eigenvectors
  // device state
  Ctl* ctl = nullptr;
  Ctl* hctl = nullptr;  // pinned mirror
  void* dbuf[3]{};
  long long dbuf_elems = 0;
  void** d_dbufs = nullptr;
  double* U[TK_MAXD]{};
  void* Uw[TK_MAXD]{};
  double* Ud[2]{};
  double** d_udbufs = nullptr;
  void* Cb[2]{};
  void* Vb[2]{};
  void** d_cbufs = nullptr;
  void** d_vbufs = nullptr;
  void* evec = nullptr;
  double* S = nullptr;
  double* Snew = nullptr;
  double* part_e2 = nullptr;
  double* part_y2 = nullptr;
  double* gpart = nullptr;
  double* G = nullptr;
  void* eAw = nullptr;
  void* eZ = nullptr;
  void* eLD = nullptr;
  double* eW = nullptr;
  double* elam = nullptr;
  double* part_p = nullptr;
  double* part_e = nullptr;
  double* pvec = nullptr;
  double* esvec = nullptr;
  SecWork sw{};
  void* Bc = nullptr;
  void* Bv = nullptr;
  float* bsplit[4]{};            // B^T TF32 hi/lo of the core and V updates (mixed form)
  float** d_bsplit = nullptr;
  TcMaps maps{};
  bool tc = false;               // tensor-core path available (mixed form)
  float* usplit[TK_MAXD][4]{};   // U_k TF32 hi/lo copies for the tensor-core spatial passes
  TcProjMaps pmaps[TK_MAXD]{};
  int tcmask = 0;                 // bit k: tensor-core projection of spatial mode k available
  void* u16[TK_MAXD][4]{};        // FP16 hi/lo parts of 2^14 U_k (U1 hi, U1 lo, U2 hi, U2 lo)
  int ld16[TK_MAXD]{};            // row stride of U1 (n_k rounded up to 64)
  int h16mask = 0;                // bit k: the FP16 pass (input tile in TMEM) runs mode k
  int blk = 1;                    // slices of the update being launched (block update)
  int block_cap = 1;              // most slices per block update (buffers sized for it)
  void* Dt = nullptr;             // block update: the projected slices as rows (R x block_cap)
  int etmask = 0;                 // bit k: tensor-core residual Gram of spatial mode k available
  float* et = nullptr;            // E^T of the growing mode (n_k x Fs_k) for the Gram
  long long et_stride[TK_MAXD]{};
  int nsm = 152;
  // launch shape of the update's kernels (tucker_set_launch_plan)
  int grid_p = kGridP;   // SIMT projection / residual passes; partial-sum slots of the norms
  int grid_tc = 152;     // tensor-core passes (one CTA per SM at most)
  int grid_i = kGridI;   // ISVD row passes
  int grid_cv = kGridCV; // core / V update
  void* cu = nullptr;
  void* wv = nullptr;
  std::vector<void*> allocs;
  // profiling
  bool prof = false;
  std::vector<cudaEvent_t> ev;       // event pool
  std::vector<int> ev_phase;         // phase of each recorded (start, end) pair
  size_t ev_used = 0;
  long long prof_launches = 0, prof_updates = 0;
  double bytes0[TK_NPH]{};
  cudaStream_t last_stream = nullptr;
  int latched = 0;
  char err[512] = "ok";
  // graph form of the update (device-side branches as conditional nodes)
  bool gform = false;                 // capturing: open an IF node around each growth chain
  bool body_open = false;
  cudaStream_t body_st = nullptr;     // captures the IF bodies
  cudaStream_t cap_st = nullptr;      // captures the single-state update graph
  cudaGraph_t ugraph = nullptr;
  cudaGraphExec_t uexec = nullptr;
  bool graph_failed = false;          // capture or instantiation failed once: stay eager
  long long graph_kernels = 0;        // kernel nodes of the update graph (bodies included)
  // graph form of block updates, one per block size (index = slices per block, 2..64)
  cudaGraph_t bgraph[65]{};
  cudaGraphExec_t bexec[65]{};
  long long bkernels[65]{};
  std::vector<cudaGraph_t> bodies;    // IF bodies created by the last capture
  // host-input updates (tucker_stream_update_host): two staging slices, a copy stream, and per
  // buffer an event after its copy and one after the update that read it
  void* hstage[2]{};
  cudaStream_t hcs = nullptr;
  cudaEvent_t hcopied[2]{}, hconsumed[2]{};
  int hnext = 0;
  // per-update log (StepRec per update) and the replay hook's pinned staging words
  StepRec* log = nullptr;
  long long log_cap = 0;
  int* rp_host = nullptr;
  bool rp_pending = false;
};

namespace {

const char* kVersion = "tucker_stream 0.2 (sm_103a)";

// rp_on, rp_grow[TK_MAXD], rp_aug: contiguous words of the control block
constexpr size_t kReplayBytes = sizeof(int) * (2 + TK_MAXD);
static_assert(offsetof(Ctl, rp_aug) == offsetof(Ctl, rp_on) + sizeof(int) * (1 + TK_MAXD), "replay words contiguous");
static_assert(sizeof(StepRec) == sizeof(tucker_step_record), "step record layout");
static_assert(offsetof(StepRec, eps) == offsetof(tucker_step_record, eps), "step record layout");
static_assert(offsetof(StepRec, discarded) == offsetof(tucker_step_record, discarded), "step record layout");

void set_err(tucker_state* s, const char* fmt, const char* a = "", long long b = 0) {
  if (!s) return;
  snprintf(s->err, sizeof(s->err), fmt, a, b);
}

#define CK(call)                                                                           \
  do {                                                                                     \
    cudaError_t e_ = (call);                                                               \
    if (e_ != cudaSuccess) {                                                               \
      set_err(s, "CUDA error: %s (line %lld)", cudaGetErrorString(e_), (long long)__LINE__); \
      return TUCKER_ECUDA;                                                                 \
    }                                                                                      \
  } while (0)

cudaError_t dalloc(tucker_state* s, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaSuccess) {
    s->allocs.push_back(*p);
    e = cudaMemset(*p, 0, bytes);
  }
  return e;
}

void free_all(tucker_state* s) {
  for (cudaEvent_t e : s->ev) cudaEventDestroy(e);
  s->ev.clear();
  for (void* p : s->allocs) cudaFree(p);
  s->allocs.clear();
  if (s->hctl) cudaFreeHost(s->hctl);
  s->hctl = nullptr;
  if (s->rp_host) cudaFreeHost(s->rp_host);
  s->rp_host = nullptr;
}

tucker_status map_status(int st) {
  switch (st) {
    case 0: return TUCKER_OK;
    case TK_ECAPACITY: return TUCKER_ECAPACITY;
    case TK_ENUMERIC: return TUCKER_ENUMERIC;
    case 5: return TUCKER_ETIMEOUT;
    default: return TUCKER_ENUMERIC;
  }
}

const char* status_msg(int st) {
  switch (st) {
    case TK_ECAPACITY: return "device: a rank, the spatial core size or n_d exceeded its capacity";
    case TK_ENUMERIC: return "device: non-finite slice norm or numerical failure";
    default: return "device: error";
  }
}

// Read the control block (synchronizes the last stream used).
tucker_status sync_ctl(tucker_state* s) {
  tucker_state* ss = s;
  {
    tucker_state* s = ss;
    CK(cudaMemcpyAsync(s->hctl, s->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, s->last_stream));
    CK(cudaStreamSynchronize(s->last_stream));
  }
  if (s->hctl->status) {
    s->latched = s->hctl->status;
    snprintf(s->err, sizeof(s->err), "%s", status_msg(s->hctl->status));
    return map_status(s->hctl->status);
  }
  return TUCKER_OK;
}

bool validate(const tucker_config* c, int64_t n_init, char* msg, size_t msz) {
  if (!c) { snprintf(msg, msz, "config is NULL"); return false; }
  if (c->ndim < 2 || c->ndim > TK_MAXD) { snprintf(msg, msz, "ndim must be in 2..8"); return false; }
  if (c->dtype != TUCKER_F32 && c->dtype != TUCKER_F64) { snprintf(msg, msz, "bad dtype"); return false; }
  if (c->precision != TUCKER_PREC_FP64 && c->precision != TUCKER_PREC_MIXED) {
    snprintf(msg, msz, "bad precision"); return false;
  }
  if (!(c->tau > 0.0) || !std::isfinite(c->tau)) { snprintf(msg, msz, "tau must be > 0"); return false; }
  if (n_init < 1 || n_init > TK_N_MAX) { snprintf(msg, msz, "n_init must be in 1..512"); return false; }
  const int spatial_cap_max = (c->precision == TUCKER_PREC_FP64) ? 256 : 512;
  for (int k = 0; k < c->ndim - 1; ++k) {
    if (c->n[k] < 1 || c->n[k] > TK_N_MAX) { snprintf(msg, msz, "n_%d must be in 1..512", k + 1); return false; }
    if (c->rank_cap[k] < 0 || c->rank_cap[k] > c->n[k]) {
      snprintf(msg, msz, "rank_cap[%d] must be in 0..n_%d", k, k + 1); return false;
    }
    const long long cap = c->rank_cap[k] ? c->rank_cap[k] : c->n[k];
    if (cap > spatial_cap_max) {
      snprintf(msg, msz, "rank_cap[%d] = %lld above %d for this precision (set a smaller cap)", k, cap,
               spatial_cap_max);
      return false;
    }
  }
  const long long scap = c->rank_cap[c->ndim - 1];
  if (scap < 0 || scap > TK_STREAM_CAP_MAX) { snprintf(msg, msz, "streaming rank cap must be <= 512"); return false; }
  if (c->steps_cap < 0 || (c->steps_cap > 0 && c->steps_cap < n_init)) {
    snprintf(msg, msz, "steps_cap must be >= n_init"); return false;
  }
  if (c->core_cap < 0) { snprintf(msg, msz, "core_cap must be >= 0"); return false; }
  if (c->block_cap < 0 || c->block_cap > 64) { snprintf(msg, msz, "block_cap must be in 0..64"); return false; }
  return true;
}

// ---------------------------------------------------------------------------------------------
// allocation
// ---------------------------------------------------------------------------------------------
tucker_status allocate(tucker_state* s, int64_t n_init) {
  const tucker_config& c = s->cfg;
  s->d = c.ndim;
  const int d = s->d;
  s->tw = (c.precision == TUCKER_PREC_MIXED) ? 4 : 8;
  s->tx = (c.dtype == TUCKER_F32) ? 4 : 8;
  s->N = 1;
  for (int k = 0; k < d - 1; ++k) {
    s->n[k] = (int)c.n[k];
    s->cap[k] = (int)(c.rank_cap[k] ? c.rank_cap[k] : c.n[k]);
    s->N *= s->n[k];
  }
  s->cap[d - 1] = (int)(c.rank_cap[d - 1] ? c.rank_cap[d - 1] : 256);
  s->ldc = s->cap[d - 1];
  s->steps_cap = (int)(c.steps_cap ? c.steps_cap : n_init + 1024);
  long long pc = 1;
  for (int k = 0; k < d - 1; ++k) pc *= s->cap[k];
  s->core_cap = c.core_cap ? c.core_cap : std::min<long long>(pc, 1LL << 22);
  s->nmax = (int)n_init;
  s->mcap = s->cap[d - 1];
  for (int k = 0; k < d - 1; ++k) {
    s->nmax = std::max(s->nmax, s->n[k]);
    s->mcap = std::max(s->mcap, s->cap[k]);
  }
  s->mcap = std::min(std::max(s->mcap, (int)n_init), TK_N_MAX);
  const int tw = s->tw;
  // D* buffers for one slice: max_k prod_{i<=k} cap_i prod_{i>k} n_i
  long long maxD = s->N;
  for (int k = 0; k < d - 1; ++k) {
    long long sz = 1;
    for (int i = 0; i < d - 1; ++i) sz *= (i <= k) ? s->cap[i] : s->n[i];
    maxD = std::max(maxD, sz);
  }
  maxD = std::max(maxD, s->core_cap);
  // a block update holds block_cap slices in flight through the spatial modes
  s->block_cap = std::max(1, (int)c.block_cap);
  s->dbuf_elems = maxD * s->block_cap;
  CK(cudaMallocHost((void**)&s->hctl, sizeof(Ctl)));
  memset(s->hctl, 0, sizeof(Ctl));
  CK(dalloc(s, (void**)&s->ctl, sizeof(Ctl)));
  s->log_cap = s->steps_cap;
  CK(dalloc(s, (void**)&s->log, sizeof(StepRec) * (size_t)s->log_cap));
  for (int i = 0; i < 3; ++i) CK(dalloc(s, &s->dbuf[i], (size_t)s->dbuf_elems * tw));
  CK(dalloc(s, (void**)&s->d_dbufs, sizeof(void*) * 3));
  CK(cudaMemcpy(s->d_dbufs, s->dbuf, sizeof(void*) * 3, cudaMemcpyHostToDevice));
  for (int k = 0; k < d - 1; ++k) {
    CK(dalloc(s, (void**)&s->U[k], sizeof(double) * s->n[k] * s->cap[k]));
    if (tw == 8) s->Uw[k] = s->U[k];
    else CK(dalloc(s, &s->Uw[k], (size_t)tw * s->n[k] * s->cap[k]));
  }
  for (int i = 0; i < 2; ++i) {
    CK(dalloc(s, (void**)&s->Ud[i], sizeof(double) * (size_t)s->steps_cap * s->ldc));
    CK(dalloc(s, &s->Cb[i], (size_t)tw * s->core_cap * s->ldc));
    CK(dalloc(s, &s->Vb[i], (size_t)tw * s->core_cap * s->ldc));
  }
  CK(dalloc(s, (void**)&s->d_udbufs, sizeof(void*) * 2));
  CK(dalloc(s, (void**)&s->d_cbufs, sizeof(void*) * 2));
  CK(dalloc(s, (void**)&s->d_vbufs, sizeof(void*) * 2));
  CK(cudaMemcpy(s->d_udbufs, s->Ud, sizeof(void*) * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_cbufs, s->Cb, sizeof(void*) * 2, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(s->d_vbufs, s->Vb, sizeof(void*) * 2, cudaMemcpyHostToDevice));
  CK(dalloc(s, &s->evec, (size_t)tw * s->core_cap));
  if (s->block_cap > 1) CK(dalloc(s, &s->Dt, (size_t)tw * s->core_cap * s->block_cap));
  CK(dalloc(s, (void**)&s->S, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&s->Snew, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&s->part_e2, sizeof(double) * 4096));
  CK(dalloc(s, (void**)&s->part_y2, sizeof(double) * 4096));
  {
    int dev0 = 0, nsm0 = 152;
    CK(cudaGetDevice(&dev0));
    CK(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev0));
    // SIMT residual Gram tiles, or the tensor-core split-K partial Grams (nsm planes of
    // n1p x n1p FP32, n_k <= 384; counted here in doubles)
    int ntc = 16;
    for (int k = 0; k < d - 1; ++k)
      if (s->n[k] <= 384) ntc = std::max(ntc, (s->n[k] + 15) / 16 * 16);
    const size_t g1 = (size_t)(kGramBlocks + 64) * 4096;
    const size_t g2 = std::max((size_t)nsm0 * 128 * 256, ((size_t)nsm0 * ntc * ntc + 1) / 2);
    CK(dalloc(s, (void**)&s->gpart, sizeof(double) * std::max(g1, g2)));
  }
  CK(dalloc(s, (void**)&s->G, sizeof(double) * (size_t)s->nmax * s->nmax));
  CK(dalloc(s, &s->eAw, sizeof(double) * (size_t)s->nmax * s->nmax));
  CK(dalloc(s, &s->eZ, sizeof(double) * (size_t)s->nmax * s->mcap));
  CK(dalloc(s, &s->eLD, sizeof(double) * (size_t)s->mcap * 2 * s->nmax));
  CK(dalloc(s, (void**)&s->eW, sizeof(double) * (size_t)s->nmax * s->mcap));
  CK(dalloc(s, (void**)&s->elam, sizeof(double) * (size_t)TK_N_MAX));
  CK(dalloc(s, (void**)&s->part_p, sizeof(double) * (size_t)kGridI * TK_STREAM_CAP_MAX));
  CK(dalloc(s, (void**)&s->part_e, sizeof(double) * (size_t)kGridI * (TK_STREAM_CAP_MAX + 2)));
  CK(dalloc(s, (void**)&s->pvec, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&s->esvec, sizeof(double) * kSecMax));
  SecWork& w = s->sw;
  CK(dalloc(s, (void**)&w.delta, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.z, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.idx, sizeof(int) * kSecMax));
  CK(dalloc(s, (void**)&w.tau, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.org, sizeof(int) * kSecMax));
  CK(dalloc(s, (void**)&w.lam, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.lsrc, sizeof(int) * kSecMax));
  CK(dalloc(s, (void**)&w.rot, sizeof(double) * 4 * kSecMax));
  CK(dalloc(s, (void**)&w.nrot, sizeof(int) * 4));
  CK(dalloc(s, (void**)&w.V2, sizeof(double) * (size_t)kSecMax * kSecMax));
  CK(dalloc(s, (void**)&w.U2, sizeof(double) * (size_t)kSecMax * kSecMax));
  CK(dalloc(s, (void**)&w.sv, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.pq, sizeof(double) * kSecMax));
  CK(dalloc(s, (void**)&w.meta, sizeof(int) * 8));
  CK(dalloc(s, &s->Bc, (size_t)tw * kSecMax * s->ldc));
  CK(dalloc(s, &s->Bv, (size_t)tw * kSecMax * s->ldc));
  CK(dalloc(s, &s->cu, (size_t)tw * kSecMax));
  CK(dalloc(s, &s->wv, (size_t)tw * kSecMax));
  int dev = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&s->nsm, cudaDevAttrMultiProcessorCount, dev));
  s->grid_tc = s->nsm;
  if (tw == 4 && s->ldc % 4 == 0) {
    for (int i = 0; i < 4; ++i) CK(dalloc(s, (void**)&s->bsplit[i], sizeof(float) * 512 * 512));
    CK(dalloc(s, (void**)&s->d_bsplit, sizeof(void*) * 4));
    CK(cudaMemcpy(s->d_bsplit, s->bsplit, sizeof(void*) * 4, cudaMemcpyHostToDevice));
    bool ok = true;
    ok &= make_map_2d_f32(&s->maps.c0, s->Cb[0], s->core_cap, s->ldc, s->ldc, 32, 128);
    ok &= make_map_2d_f32(&s->maps.c1, s->Cb[1], s->core_cap, s->ldc, s->ldc, 32, 128);
    ok &= make_map_2d_f32(&s->maps.v0, s->Vb[0], s->core_cap, s->ldc, s->ldc, 32, 128);
    ok &= make_map_2d_f32(&s->maps.v1, s->Vb[1], s->core_cap, s->ldc, s->ldc, 32, 128);
    ok &= make_map_2d_f32(&s->maps.bc_hi, s->bsplit[0], 512, 512, 512, 32, 16);
    ok &= make_map_2d_f32(&s->maps.bc_lo, s->bsplit[1], 512, 512, 512, 32, 16);
    ok &= make_map_2d_f32(&s->maps.bv_hi, s->bsplit[2], 512, 512, 512, 32, 16);
    ok &= make_map_2d_f32(&s->maps.bv_lo, s->bsplit[3], 512, 512, 512, 32, 16);
    s->tc = ok;
  }
  if (tw == 4) {
    // tensor-core spatial passes: per mode, TF32 splits of U_k and the tensor maps.
    // E^T rows have stride Fs_k >= max fibers + 32, so a Gram K chunk never leaves its row.
    size_t et_elems = 16;
    for (int k = 0; k < d - 1; ++k) {
      const long long fs = (s->dbuf_elems / s->n[k] + 32 + 3) / 4 * 4;
      et_elems = std::max(et_elems, (size_t)fs * s->n[k]);
    }
    CK(dalloc(s, (void**)&s->et, sizeof(float) * et_elems));
    for (int k = 0; k < d - 1; ++k) {
      const int nk = s->n[k];
      if (nk % 4 != 0 || nk > 512 || (k == 0 && s->tx != 4)) continue;
      for (int i = 0; i < 2; ++i) CK(dalloc(s, (void**)&s->usplit[k][i], sizeof(float) * nk * s->cap[k]));
      for (int i = 2; i < 4; ++i) CK(dalloc(s, (void**)&s->usplit[k][i], sizeof(float) * nk * 64));
      TcProjMaps& m = s->pmaps[k];
      bool ok = true;
      ok &= make_map_2d_f32(&m.uhi, s->usplit[k][0], s->cap[k], nk, nk, 32, 16);
      ok &= make_map_2d_f32(&m.ulo, s->usplit[k][1], s->cap[k], nk, nk, 32, 16);
      ok &= make_map_2d_f32(&m.urhi, s->usplit[k][2], nk, 64, 64, 32, 16);
      ok &= make_map_2d_f32(&m.urlo, s->usplit[k][3], nk, 64, 64, 32, 16);
      const long long rows = s->dbuf_elems / nk;
      for (int i = 0; i < 3; ++i) ok &= make_map_2d_f32(&m.d[i], s->dbuf[i], rows, nk, nk, 32, 128);
      if (!ok) continue;
      s->tcmask |= 1 << k;
      if (nk <= TK_H16_NMAX) {
        const int ld1 = (nk + 63) / 64 * 64;
        s->ld16[k] = ld1;
        for (int i = 0; i < 2; ++i) CK(dalloc(s, &s->u16[k][i], 2 * (size_t)TP_RMAX * ld1));
        for (int i = 2; i < 4; ++i) CK(dalloc(s, &s->u16[k][i], 2 * (size_t)nk * TP_RMAX));
        bool okh = make_map_2d_f16(&m.h1hi, s->u16[k][0], TP_RMAX, nk, ld1, 64, 16);
        okh &= make_map_2d_f16(&m.h1lo, s->u16[k][1], TP_RMAX, nk, ld1, 64, 16);
        okh &= make_map_2d_f16(&m.h2hi, s->u16[k][2], nk, TP_RMAX, TP_RMAX, 64, 64);
        okh &= make_map_2d_f16(&m.h2lo, s->u16[k][3], nk, TP_RMAX, TP_RMAX, 64, 64);
        if (okh) s->h16mask |= 1 << k;
      }
      const long long fs = (s->dbuf_elems / nk + 32 + 3) / 4 * 4;
      s->et_stride[k] = fs;
      // the tensor-core residual Gram takes n_k <= 384 (three 128-row blocks)
      bool oke = nk <= 384 && make_map_2d_f32(&m.eta, s->et, nk, fs, fs, 32, 128);
      if (oke) s->etmask |= 1 << k;
    }
  }
  return TUCKER_OK;
}

// Phase markers: with profiling on, record an event pair around each phase on the stream.
struct PhaseMark {
  tucker_state* s;
  cudaStream_t st;
  int phase;
  size_t idx;
  // ph < 0: no mark
  PhaseMark(tucker_state* s_, cudaStream_t st_, int ph) : s(s_), st(st_), phase(ph), idx(0) {
    if (!s->prof || ph < 0) return;
    while (s->ev.size() < s->ev_used + 2) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      s->ev.push_back(e);
    }
    idx = s->ev_used;
    s->ev_used += 2;
    s->ev_phase.push_back(phase);
    cudaEventRecord(s->ev[idx], st);
  }
  ~PhaseMark() {
    if (s->prof && phase >= 0) cudaEventRecord(s->ev[idx + 1], st);
  }
};

int gram_pairs(int n) {
  const int T = (n + 63) / 64;
  return T * (T + 1) / 2;
}
int gram_chunks(int n) { return std::max(1, kGramBlocks / gram_pairs(n)); }

// ---------------------------------------------------------------------------------------------
// batch ST-HOSVD (Alg. 2) on the device
// ---------------------------------------------------------------------------------------------
// Tensor-core copies of U_k after it changed (pred: only if mode k grew in this update).
cudaError_t split_u(tucker_state* s, int k, int pred, cudaStream_t st) {
  if ((s->h16mask >> k) & 1)
    return launch_split_u16(s->ctl, k, pred, s->U[k], s->n[k], s->ld16[k], s->u16[k], st);
  return launch_split_u(s->ctl, k, pred, s->U[k], s->n[k], s->usplit[k], st);
}

// Mode k's tensor-core pass (mode 0 projection, 1 projection + residual norms, 2 residual E^T):
// the FP16 form where it applies, else the 3xTF32 form. rerun = 1: the second launch of the FP16
// form's pass A, which runs the pass again only if its input left the FP16 scale window (nothing
// to launch for the 3xTF32 form).
cudaError_t tc_pass(tucker_state* s, int k, int mode, int pred, int rerun, const void* Y,
                    int out_off, double* part_e2, double* part_y2, float* Et, long long et_stride,
                    cudaStream_t st) {
  const long long F0 = s->N / s->n[0] * s->blk;
  if ((s->h16mask >> k) & 1)
    return launch_tc_pass16(s->ctl, k, mode, pred, rerun, (const float*)Y, F0, s->n[0],
                            s->pmaps[k], s->d_dbufs, out_off, part_e2, part_y2, s->grid_p, Et,
                            et_stride, s->grid_tc, st);
  if (rerun) return cudaSuccess;
  return launch_tc_proj(s->ctl, k, mode, pred, (const float*)Y, F0, s->n[0], s->pmaps[k],
                        s->d_dbufs, out_off, part_e2, part_y2, s->grid_p, Et, et_stride,
                        s->grid_tc, st);
}

template <typename TX, typename TW, typename TE>
tucker_status do_init(tucker_state* s, const void* X, int64_t n_init, cudaStream_t st) {
  const int d = s->d;
  Ctl& h = *s->hctl;
  memset(&h, 0, sizeof(Ctl));
  h.d = d;
  for (int k = 0; k < d - 1; ++k) { h.n[k] = s->n[k]; h.r[k] = s->n[k]; }
  for (int k = 0; k < d; ++k) h.cap[k] = s->cap[k];
  h.r[d - 1] = (int)n_init;
  h.core_cap = s->core_cap;
  h.steps_cap = s->steps_cap;
  h.ldc = s->ldc;
  h.tau = s->cfg.tau;
  h.eps_m = s->cfg.eps_m > 0 ? s->cfg.eps_m : 1e-10;
  h.xbuf = -1;
  h.init_nt = (int)n_init;
  h.tx = s->tx;
  h.tw = s->tw;
  h.N = s->N;
  h.tcmask = s->tcmask;
  h.etmask = s->etmask;
  h.log = s->log;
  h.log_cap = s->log_cap;
  // ||X||^2 -> eps (Alg. 2, first step)
  const long long NX = s->N * n_init;
  CK(launch_norm2<TX>(X, NX, s->part_y2, 1024, st));
  std::vector<double> parts(1024);
  CK(cudaMemcpyAsync(parts.data(), s->part_y2, sizeof(double) * 1024, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double x2 = 0.0;
  for (double v : parts) x2 += v;
  if (!std::isfinite(x2)) { set_err(s, "initial data is not finite"); return TUCKER_ENUMERIC; }
  if (x2 == 0.0) { set_err(s, "initial data is all zero (Assumption 1(c) needs S > 0)"); return TUCKER_EINVAL; }
  h.eps = s->cfg.tau * std::sqrt(x2) / std::sqrt((double)d);
  h.data2 = x2;
  {
    // first FP16 scale of every mode's input: from the norm of an average initial slice (an
    // upper bound of its entries; the first update re-scales a mode whose input lies far below)
    int e2 = 0;
    std::frexp(std::sqrt(x2 / (double)n_init), &e2);
    for (int k = 0; k < TK_MAXD; ++k) h.x16e[k] = x16_sigma_for(e2 - 1);
  }
  h.y2 = x2;
  CK(cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st));
  // temporary partial-core buffers (the initial slices are larger than one slice)
  void* ib[3] = {nullptr, nullptr, nullptr};
  void** d_ib = nullptr;
  const size_t ibytes = (size_t)s->tw * (size_t)NX;
  auto cleanup = [&]() {
    for (int i = 0; i < 3; ++i) if (ib[i]) cudaFree(ib[i]);
    if (d_ib) cudaFree(d_ib);
  };
  for (int i = 0; i < 3; ++i) {
    if (cudaMalloc(&ib[i], ibytes) != cudaSuccess) { cleanup(); set_err(s, "out of device memory (initial ST-HOSVD buffers)"); return TUCKER_ENOMEM; }
  }
  if (cudaMalloc((void**)&d_ib, sizeof(void*) * 3) != cudaSuccess) { cleanup(); return TUCKER_ENOMEM; }
  cudaMemcpy(d_ib, ib, sizeof(void*) * 3, cudaMemcpyHostToDevice);
  double* Utmp = nullptr;
  void* Uwtmp = nullptr;
  cudaMalloc((void**)&Utmp, sizeof(double) * n_init * s->cap[d - 1]);
  cudaMalloc(&Uwtmp, (size_t)s->tw * n_init * s->cap[d - 1]);
  auto cleanup2 = [&]() { cleanup(); cudaFree(Utmp); cudaFree(Uwtmp); };
  tucker_status rc = TUCKER_OK;
  for (int k = 0; k < d && rc == TUCKER_OK; ++k) {
    const int nv = (k == d - 1) ? (int)n_init : s->n[k];
    const int pairs = gram_pairs(nv), chunks = gram_chunks(nv);
    cudaError_t e;
    if (k == 0) e = launch_resid_gram<TX, double>(s->ctl, k, nv, X, d_ib, nullptr, 0, s->gpart, pairs, chunks, 1, st);
    else e = launch_resid_gram<TW, double>(s->ctl, k, nv, X, d_ib, nullptr, 0, s->gpart, pairs, chunks, 1, st);
    if (e == cudaSuccess) e = launch_gram_reduce(s->ctl, k, s->gpart, pairs, chunks, s->G, 1, st);
    if (e == cudaSuccess) e = launch_eig<double>(s->ctl, k, 1, s->G, s->eAw, s->eZ, s->eLD, s->eW, s->elam, s->mcap, nv, st);
    double* Uk = (k == d - 1) ? Utmp : s->U[k];
    void* Uwk = (k == d - 1) ? (s->tw == 8 ? (void*)Utmp : Uwtmp) : s->Uw[k];
    if (e == cudaSuccess) e = launch_append<TW>(s->ctl, k, 1, s->eW, Uk, (s->tw == 8) ? nullptr : Uwk, nv, nv, st);
    if (e == cudaSuccess && k < d - 1 && ((s->tcmask >> k) & 1)) e = split_u(s, k, 0, st);
    if (e != cudaSuccess) { set_err(s, "CUDA error (%s) in the Gram/eig/append step of mode %lld", cudaGetErrorString(e), k + 1); rc = TUCKER_ECUDA; break; }
    s->last_stream = st;
    rc = sync_ctl(s);
    if (rc != TUCKER_OK) break;
    const int rk = s->hctl->r[k];
    if (k == d - 2) {
      long long R = 1;
      for (int i = 0; i < d - 1; ++i) R *= s->hctl->r[i];
      if (R > s->core_cap) { set_err(s, "spatial core size %s%lld exceeds core_cap", "", R); rc = TUCKER_ECAPACITY; break; }
    }
    if (k == 0) e = launch_proj<TX, TW>(s->ctl, k, 1, 0, X, d_ib, Uwk, nv, rk, nullptr, nullptr, kGridP, st);
    else e = launch_proj<TW, TW>(s->ctl, k, 1, 0, X, d_ib, Uwk, nv, rk, nullptr, nullptr, kGridP, st);
    if (e == cudaSuccess) e = launch_mode_end(s->ctl, k, 0, st);
    if (e != cudaSuccess) { set_err(s, "CUDA error (%s) in the projection of mode %lld", cudaGetErrorString(e), k + 1); rc = TUCKER_ECUDA; break; }
  }
  if (rc == TUCKER_OK) rc = sync_ctl(s);
  if (rc == TUCKER_OK) {
    Ctl& c = *s->hctl;
    long long R = 1;
    for (int i = 0; i < d - 1; ++i) R *= c.r[i];
    const int rd = c.r[d - 1];
    cudaError_t e = launch_init_finish<TW>(s->ctl, ib[c.xbuf], R, rd, s->elam, Utmp, (int)n_init, s->Cb[0], s->Vb[0],
                                           s->Ud[0], s->S, s->ldc, st);
    if (e == cudaSuccess && s->tw == 4) {
      // mixed form: C_(d)^T = C*_{d-1} U_d again in FP64 (U_d row-major in Ud[0] now), and C, V
      // from it; C*_{d-1} is the buffer before the last mode's output
      double* C64 = nullptr;
      e = cudaMalloc((void**)&C64, sizeof(double) * (size_t)R * rd);
      if (e == cudaSuccess)
        e = launch_expand<float, double, double>(ib[(c.xbuf + 2) % 3], R, (int)n_init, 1, s->Ud[0], s->ldc, rd, C64, st);
      if (e == cudaSuccess) e = launch_init_cv64<float>(C64, R, rd, s->elam, s->Cb[0], s->Vb[0], s->ldc, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (C64) cudaFree(C64);
    }
    if (e != cudaSuccess) { set_err(s, "CUDA error (%s) in the core factorization (R = %lld)", cudaGetErrorString(e), R); rc = TUCKER_ECUDA; }
    if (rc == TUCKER_OK) {
      double err2 = 0.0;
      for (int k = 0; k < d; ++k) err2 += c.disc[k];
      c.err2 = err2;
      c.data2 = x2;
      c.nd = (int)n_init;
      c.init_nt = 0;
      c.xbuf = -1;
      c.cbuf = 0;
      c.ubuf = 0;
      for (int k = 0; k < TK_MAXD; ++k) { c.grew[k] = 0; c.radd[k] = 0; c.disc[k] = 0.0; c.rold[k] = c.r[k]; }
      if (cudaMemcpyAsync(s->ctl, &c, sizeof(Ctl), cudaMemcpyHostToDevice, st) != cudaSuccess ||
          cudaStreamSynchronize(st) != cudaSuccess) { rc = TUCKER_ECUDA; set_err(s, "CUDA error after init"); }
    }
  }
  cleanup2();
  return rc;
}

// ---------------------------------------------------------------------------------------------
// graph form: an IF node (condition set on the device) around a chain of launches
// ---------------------------------------------------------------------------------------------
cudaError_t cond_handle(cudaStream_t st, cudaGraphConditionalHandle* h) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, nullptr, nullptr, nullptr);
  if (e != cudaSuccess) return e;
  if (cs != cudaStreamCaptureStatusActive) return cudaErrorStreamCaptureInvalidated;
  // the condition is 0 at every launch unless a kernel sets it
  return cudaGraphConditionalHandleCreate(h, g, 0, cudaGraphCondAssignDefault);
}

// Appends the IF node to the capture of st and starts capturing its body on body_st (the body
// graph is appended to `bodies`).
cudaError_t cond_begin(cudaStream_t st, cudaStream_t body_st, cudaGraphConditionalHandle h,
                       std::vector<cudaGraph_t>* bodies) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t g = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(st, &cs, nullptr, &g, &deps, nullptr, &nd);
  if (e != cudaSuccess) return e;
  cudaGraphNodeParams p{};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, g, deps, nullptr, nd, &p);
  if (e != cudaSuccess) return e;
  e = cudaStreamUpdateCaptureDependencies(st, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
  if (e != cudaSuccess) return e;
  if (bodies) bodies->push_back(p.conditional.phGraph_out[0]);
  return cudaStreamBeginCaptureToGraph(body_st, p.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                       cudaStreamCaptureModeThreadLocal);
}

cudaError_t cond_end(cudaStream_t body_st) {
  cudaGraph_t g = nullptr;
  return cudaStreamEndCapture(body_st, &g);
}

// Kernel nodes directly in g (the bodies of its conditional nodes are separate graphs).
long long count_kernel_nodes(cudaGraph_t g) {
  size_t nn = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) return 0;
  std::vector<cudaGraphNode_t> nodes(nn);
  if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return 0;
  long long c = 0;
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(nd, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++c;
  }
  return c;
}

// ---------------------------------------------------------------------------------------------
// streaming update (Alg. 5): fixed launch sequence, device-side branches
// ---------------------------------------------------------------------------------------------
template <typename TX, typename TW, typename TE>
tucker_status do_update(tucker_state* s, const void* Y, cudaStream_t st) {
  const int d = s->d;
  long long launches = 0;
  // (an IF node costs more than the empty launch of a predicated kernel on this GPU, so only the
  // 11-kernel growth chains below are conditional nodes)
  CK(launch_begin(s->ctl, st, s->blk));
  launches += 1;
  for (int k = 0; k < d - 1; ++k) {
    const int n = s->n[k];
    const int pairs = gram_pairs(n), chunks = gram_chunks(n);
    const bool tck = (s->tcmask >> k) & 1;
    {
      // pass A: P_k = D*_{k-1} x_k U_k^T, ||E_k||^2 (and ||Y||^2 for k = 0); Alg. 4's branch
      PhaseMark pm(s, st, k == 0 ? TK_PH_PROJ1 : TK_PH_PROJN);
      if (tck) {
        {
          PhaseMark pk(s, st, k == 0 ? TK_PH_SLICE : -1);
          CK(tc_pass(s, k, 1, 0, 0, Y, 1, s->part_e2, k == 0 ? s->part_y2 : nullptr, nullptr, 0, st));
        }
        CK(tc_pass(s, k, 1, 0, 1, Y, 1, s->part_e2, k == 0 ? s->part_y2 : nullptr, nullptr, 0, st));
        launches += ((s->h16mask >> k) & 1) ? 2 : 1;
      }
      if (k == 0) {
        PhaseMark pk(s, st, tck ? -1 : TK_PH_SLICE);
        CK((launch_proj<TX, TW>(s->ctl, k, 1, 0, Y, s->d_dbufs, s->Uw[k], n, s->cap[k], s->part_e2,
                                s->part_y2, s->grid_p, st)));
      }
      else
        CK((launch_proj<TW, TW>(s->ctl, k, 1, 0, Y, s->d_dbufs, s->Uw[k], n, s->cap[k], s->part_e2,
                                nullptr, s->grid_p, st)));
      cudaGraphConditionalHandle hc = 0;
      if (s->gform) CK(cond_handle(st, &hc));
      CK(launch_decide(s->ctl, k, s->part_e2, s->part_y2, s->grid_p, hc, st));
      if (s->gform) {
        // graph form: the growth chain below is the body of an IF node on grew[k]
        CK(cond_begin(st, s->body_st, hc, &s->bodies));
        s->body_open = true;
      }
    }
    {
      // ||E_k|| > eps: residual Gram, eig + rank cut (Alg. 1), augmentation, then
      // pass C: D*_k = D*_{k-1} x_k U~_k^T (= Concatenate(P_k, L_k), App. C)
      const cudaStream_t main_st = st;
      cudaStream_t st = s->gform ? s->body_st : main_st;
      PhaseMark pm(s, st, TK_PH_GROW);
      if ((s->etmask >> k) & 1) {
        // residual E^T of mode k, then its Gram on the tensor cores (only if mode k grew)
        CK(tc_pass(s, k, 2, 1, 0, Y, 1, nullptr, nullptr, s->et, s->et_stride[k], st));
        CK(launch_tc_gram(s->ctl, k, s->pmaps[k], n, s->gpart, s->G, s->grid_tc, st));
        launches += 3;
      }
      if (k == 0)
        CK((launch_resid_gram<TX, TW>(s->ctl, k, n, Y, s->d_dbufs, s->Uw[k], n, s->gpart, pairs,
                                      chunks, 0, st)));
      else
        CK((launch_resid_gram<TW, TW>(s->ctl, k, n, Y, s->d_dbufs, s->Uw[k], n, s->gpart, pairs,
                                      chunks, 0, st)));
      CK(launch_gram_reduce(s->ctl, k, s->gpart, pairs, chunks, s->G, 0, st));
      if (sizeof(TE) == 4) {
        // mixed form: subspace iteration with the cut in FP64; the full FP32 tridiagonal solver
        // only where that cannot certify the cut
        CK(launch_eig_sub(s->ctl, k, s->G, s->eAw, s->eW, s->mcap, s->gpart, n, st));
        CK(launch_eig<TE>(s->ctl, k, 2, s->G, s->eAw, s->eZ, s->eLD, s->eW, nullptr, s->mcap, n, st));
        CK(launch_eig_refine_post(s->ctl, k, s->G, s->eW, s->mcap, s->gpart, n, st));
        launches += 3;
      } else {
        CK(launch_eig<TE>(s->ctl, k, 0, s->G, s->eAw, s->eZ, s->eLD, s->eW, nullptr, s->mcap, n, st));
      }
      CK(launch_append<TW>(s->ctl, k, 0, s->eW, s->U[k], (s->tw == 8) ? nullptr : s->Uw[k], n, n, st));
      if (tck) {
        CK(split_u(s, k, 1, st));
        CK(tc_pass(s, k, 0, 1, 0, Y, 2, nullptr, nullptr, nullptr, 0, st));
        launches += 2;
      }
      if (k == 0)
        CK((launch_proj<TX, TW>(s->ctl, k, 2, 1, Y, s->d_dbufs, s->Uw[k], n, s->cap[k], nullptr,
                                nullptr, s->grid_p, st)));
      else
        CK((launch_proj<TW, TW>(s->ctl, k, 2, 1, Y, s->d_dbufs, s->Uw[k], n, s->cap[k], nullptr,
                                nullptr, s->grid_p, st)));
      CK(launch_mode_end(s->ctl, k, 1, st));
      if (s->gform) {
        CK(cond_end(s->body_st));
        s->body_open = false;
      }
    }
    launches += 8;
  }
  // block update: the projected slices become rows, one incremental-SVD step each
  const int nrows = s->blk;
  if (nrows > 1) {
    CK(launch_block_rows<TW>(s->ctl, s->d_dbufs, s->Dt, st));
    launches += 1;
  }
  for (int row = 0; row < nrows; ++row) {
    if (nrows > 1) {
      CK(launch_row_begin<TW>(s->ctl, row, s->d_dbufs, s->Dt, st));
      launches += 1;
    }
    {
      // streaming mode: incremental SVD (Alg. 3)
      PhaseMark pm(s, st, TK_PH_ISVD);
      CK(launch_isvd<TW>(s->ctl, s->d_dbufs, s->d_vbufs, s->part_p, s->part_e, s->pvec, s->esvec,
                         s->evec, s->S, s->sw, s->grid_i, st));
      CK(launch_secular_vectors(s->ctl, s->S, s->sw, s->Snew, st));
      launches += 6;
    }
    {
      PhaseMark pm(s, st, TK_PH_FACT);
      CK(launch_factor<TW>(s->ctl, s->d_udbufs, s->sw, s->esvec, s->Bc, s->cu, s->Bv, s->wv, s->ldc,
                           s->tc ? s->d_bsplit : nullptr, 152 * 2, st));
      launches += 2;
    }
    {
      // core update (Alg. 5, last step) and V~ = V' V''
      PhaseMark pm(s, st, TK_PH_CV);
      if (s->tc) {
        CK(launch_tc_cv(s->ctl, s->sw, s->maps, s->Cb, s->Vb, s->d_cbufs, s->d_vbufs, s->cu, s->wv,
                        s->evec, s->d_dbufs, s->ldc, s->grid_tc, st));
        launches += 3;
      }
      CK(launch_cv<TW>(s->ctl, s->d_dbufs, s->d_cbufs, s->d_vbufs, s->sw, s->Bc, s->cu, s->Bv, s->wv,
                       s->ldc, s->evec, s->grid_cv, st));
      launches += 2;
    }
    CK(launch_end(s->ctl, s->Snew, s->S, st));
    launches += 1;
  }
  if (s->prof) {
    s->prof_launches += launches;
    s->prof_updates += 1;
  }
  return TUCKER_OK;
}

template <typename TW>
tucker_status do_reconstruct(tucker_state* s, int64_t t0, int64_t t1, void* out, cudaStream_t st) {
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  const int d = s->d;
  const long long T = t1 - t0;
  long long R = 1;
  for (int i = 0; i < d - 1; ++i) R *= c.r[i];
  const int rd = c.r[d - 1];
  const long long big = s->N * T;
  void* tmp[2] = {nullptr, nullptr};
  CK(cudaMallocAsync(&tmp[0], (size_t)s->tw * std::max(big, R * T), st));
  CK(cudaMallocAsync(&tmp[1], (size_t)s->tw * std::max(big, R * T), st));
  CK(launch_core_times_ud<TW>(s->Cb[c.cbuf], R, rd, s->ldc, s->Ud[c.ubuf], t0, T, tmp[0], st));
  int cur = 0;
  for (int k = 0; k < d - 1; ++k) {
    long long A = 1, B = T;
    for (int i = 0; i < k; ++i) A *= s->n[i];
    for (int i = k + 1; i < d - 1; ++i) B *= c.r[i];
    const bool last = (k == d - 2);
    void* dst = last ? out : tmp[cur ^ 1];
    cudaError_t e;
    if (s->tw == 4) {
      if (last && s->tx == 8) e = launch_expand<float, float, double>(tmp[cur], A, c.r[k], B, s->Uw[k], s->n[k], s->n[k], dst, st);
      else e = launch_expand<float, float, float>(tmp[cur], A, c.r[k], B, s->Uw[k], s->n[k], s->n[k], dst, st);
    } else {
      if (last && s->tx == 4) e = launch_expand<double, double, float>(tmp[cur], A, c.r[k], B, s->U[k], s->n[k], s->n[k], dst, st);
      else e = launch_expand<double, double, double>(tmp[cur], A, c.r[k], B, s->U[k], s->n[k], s->n[k], dst, st);
    }
    CK(e);
    cur ^= 1;
  }
  CK(cudaFreeAsync(tmp[0], st));
  CK(cudaFreeAsync(tmp[1], st));
  return TUCKER_OK;
}

bool usable(tucker_state* s) { return s && !s->latched; }

// ---------------------------------------------------------------------------------------------
// allocation-free reconstruction: the two ping-pong temporaries live in one fixed device array
// ---------------------------------------------------------------------------------------------
constexpr size_t kNoallocScratchBytes = (size_t)TUCKER_NOALLOC_SCRATCH_BYTES;

}  // namespace

// Every GPU that loads this library holds this array until the process exits. Host code must not
// use its name as a device address: the device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[TUCKER_NOALLOC_SCRATCH_BYTES];

namespace {

// Device address of g_noalloc_scratch in the current device's context. Looked up on every call
// (the lookup allocates nothing): a cached address would dangle once the context is recreated
// (after cudaDeviceReset, for instance). The first lookup in a context loads the module's
// device symbols, which is why the first call on a device belongs outside any stream capture.
tucker_status noalloc_scratch(tucker_state* s, void** out) {
  *out = nullptr;
  void* p = nullptr;
  CK(cudaGetSymbolAddress(&p, g_noalloc_scratch));
  *out = p;
  return TUCKER_OK;
}

// Same launch sequence as do_reconstruct; the temporaries are the two halves of the fixed array.
template <typename TW>
tucker_status do_reconstruct_noalloc(tucker_state* s, int64_t t0, int64_t t1, void* out,
                                     cudaStream_t st) {
  const Ctl& c = *s->hctl;
  const int d = s->d;
  const long long T = t1 - t0;
  long long R = 1;
  for (int i = 0; i < d - 1; ++i) R *= c.r[i];
  const int rd = c.r[d - 1];
  // largest temporary: C x_d U_d(t0:t1, :) (R x T), then every partial expansion but the last
  long long need = R * T;
  for (int k = 0; k + 1 < d - 1; ++k) {
    long long e = T;
    for (int i = 0; i <= k; ++i) e *= s->n[i];
    for (int i = k + 1; i < d - 1; ++i) e *= c.r[i];
    need = std::max(need, e);
  }
  const size_t half = kNoallocScratchBytes / 2;
  if ((size_t)need * (size_t)s->tw > half) {
    snprintf(s->err, sizeof(s->err),
             "tucker_reconstruct_noalloc: slices [%lld, %lld) need %lld bytes per temporary, above "
             "the fixed %zu-byte half of the scratch array; reconstruct fewer slices per call",
             (long long)t0, (long long)t1, need * (long long)s->tw, half);
    return TUCKER_EINVAL;
  }
  void* base = nullptr;
  tucker_status rc = noalloc_scratch(s, &base);
  if (rc != TUCKER_OK) return rc;
  void* tmp[2] = {base, (void*)((unsigned char*)base + half)};
  CK(launch_core_times_ud<TW>(s->Cb[c.cbuf], R, rd, s->ldc, s->Ud[c.ubuf], t0, T, tmp[0], st));
  int cur = 0;
  for (int k = 0; k < d - 1; ++k) {
    long long A = 1, B = T;
    for (int i = 0; i < k; ++i) A *= s->n[i];
    for (int i = k + 1; i < d - 1; ++i) B *= c.r[i];
    const bool last = (k == d - 2);
    void* dst = last ? out : tmp[cur ^ 1];
    cudaError_t e;
    if (s->tw == 4) {
      if (last && s->tx == 8) e = launch_expand<float, float, double>(tmp[cur], A, c.r[k], B, s->Uw[k], s->n[k], s->n[k], dst, st);
      else e = launch_expand<float, float, float>(tmp[cur], A, c.r[k], B, s->Uw[k], s->n[k], s->n[k], dst, st);
    } else {
      if (last && s->tx == 4) e = launch_expand<double, double, float>(tmp[cur], A, c.r[k], B, s->U[k], s->n[k], s->n[k], dst, st);
      else e = launch_expand<double, double, double>(tmp[cur], A, c.r[k], B, s->U[k], s->n[k], s->n[k], dst, st);
    }
    CK(e);
    cur ^= 1;
  }
  return TUCKER_OK;
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// batched form: one update of many independent states captured as one CUDA graph
// ---------------------------------------------------------------------------------------------
struct tucker_batch {
  std::vector<tucker_state*> states;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;   // kernel nodes per graph launch
  char err[256] = "ok";
};

namespace {

tucker_status update_dispatch(tucker_state* s, const void* Y, cudaStream_t st) {
  const bool mixed = s->cfg.precision == TUCKER_PREC_MIXED;
  const bool f32 = s->cfg.dtype == TUCKER_F32;
  if (mixed) return f32 ? do_update<float, float, float>(s, Y, st) : do_update<double, float, float>(s, Y, st);
  return f32 ? do_update<float, double, double>(s, Y, st) : do_update<double, double, double>(s, Y, st);
}

tucker_status ensure_streams(tucker_state* s) {
  if (!s->cap_st) CK(cudaStreamCreateWithFlags(&s->cap_st, cudaStreamNonBlocking));
  if (!s->body_st) CK(cudaStreamCreateWithFlags(&s->body_st, cudaStreamNonBlocking));
  return TUCKER_OK;
}

// One update of s (blk slices: 1 for Alg. 5, more for a block update), slice read from the
// control block's slot, captured as a CUDA graph whose growth chains are IF nodes on grew[k]
// (set by k_decide).
tucker_status capture_update(tucker_state* s, int blk, cudaGraph_t* graph, cudaGraphExec_t* exec,
                             long long* kernels) {
  tucker_status rc = ensure_streams(s);
  if (rc != TUCKER_OK) return rc;
  s->bodies.clear();
  CK(cudaStreamBeginCapture(s->cap_st, cudaStreamCaptureModeThreadLocal));
  const bool prof = s->prof;
  s->prof = false;
  s->gform = true;
  s->blk = blk;
  rc = update_dispatch(s, nullptr, s->cap_st);
  s->blk = 1;
  s->gform = false;
  s->prof = prof;
  if (s->body_open) {
    cudaGraph_t gb = nullptr;
    cudaStreamEndCapture(s->body_st, &gb);
    s->body_open = false;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(s->cap_st, &g);
  if (rc != TUCKER_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != TUCKER_OK ? rc : TUCKER_ECUDA;
  }
  if (cudaGraphInstantiate(exec, g, 0) != cudaSuccess) {
    *exec = nullptr;
    cudaGraphDestroy(g);
    cudaGetLastError();
    return TUCKER_ECUDA;
  }
  *graph = g;
  *kernels = count_kernel_nodes(g);
  for (cudaGraph_t b : s->bodies) *kernels += count_kernel_nodes(b);
  s->bodies.clear();
  return TUCKER_OK;
}

// Drop every captured update graph of s (launch shapes changed, or the state is destroyed).
void drop_graphs(tucker_state* s) {
  if (s->uexec) { cudaGraphExecDestroy(s->uexec); s->uexec = nullptr; }
  if (s->ugraph) { cudaGraphDestroy(s->ugraph); s->ugraph = nullptr; }
  s->graph_kernels = 0;
  for (int b = 0; b < 65; ++b) {
    if (s->bexec[b]) { cudaGraphExecDestroy(s->bexec[b]); s->bexec[b] = nullptr; }
    if (s->bgraph[b]) { cudaGraphDestroy(s->bgraph[b]); s->bgraph[b] = nullptr; }
    s->bkernels[b] = 0;
  }
}

// Capture: origin stream -> fork event -> one branch stream per state (its whole update) ->
// join events -> origin. Streams and events exist only during the capture.
tucker_status capture_batch(tucker_batch* b, const void* const* Y, cudaStream_t* streams,
                            cudaEvent_t* evs) {
  const int count = (int)b->states.size();
  cudaStream_t origin = streams[count];
  if (cudaStreamBeginCapture(origin, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return TUCKER_ECUDA;
  tucker_status rc = TUCKER_OK;
  if (cudaEventRecord(evs[count], origin) != cudaSuccess) rc = TUCKER_ECUDA;
  for (int i = 0; i < count && rc == TUCKER_OK; ++i) {
    tucker_state* s = b->states[i];
    if (cudaStreamWaitEvent(streams[i], evs[count], 0) != cudaSuccess) { rc = TUCKER_ECUDA; break; }
    const bool prof = s->prof;
    rc = ensure_streams(s);
    if (rc != TUCKER_OK) break;
    s->prof = false;
    s->gform = true;
    s->bodies.clear();
    rc = update_dispatch(s, Y[i], streams[i]);
    s->gform = false;
    s->prof = prof;
    if (s->body_open) {
      cudaGraph_t gb = nullptr;
      cudaStreamEndCapture(s->body_st, &gb);
      s->body_open = false;
    }
    if (rc != TUCKER_OK) {
      snprintf(b->err, sizeof(b->err), "state %d: %s", i, s->err);
      break;
    }
    if (cudaEventRecord(evs[i], streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(origin, evs[i], 0) != cudaSuccess) rc = TUCKER_ECUDA;
  }
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(origin, &g);
  if (rc != TUCKER_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    if (rc == TUCKER_OK) rc = TUCKER_ECUDA;
    return rc;
  }
  b->graph = g;
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) return TUCKER_ECUDA;
  b->launches = count_kernel_nodes(g);
  for (tucker_state* s : b->states) {
    for (cudaGraph_t bg : s->bodies) b->launches += count_kernel_nodes(bg);
    s->bodies.clear();
  }
  return TUCKER_OK;
}

// The replay hook's forced decisions (tucker_replay_next) go into the control block on the
// stream of the update they apply to.
tucker_status push_replay(tucker_state* s, cudaStream_t st) {
  if (!s->rp_pending) return TUCKER_OK;
  s->rp_pending = false;
  CK(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(s->ctl) + offsetof(Ctl, rp_on), s->rp_host,
                     kReplayBytes, cudaMemcpyHostToDevice, st));
  return TUCKER_OK;
}

// Graph-form slice slot: the slice's address (and, for the tensor-core mode-1 pass, its TMA
// descriptor over the blk slices' mode-1 fibers) written into the control block by a one-block
// kernel on `st`.
tucker_status write_slot(tucker_state* s, const void* Y_dev, cudaStream_t st, int blk = 1) {
  SlotArgs sa{};
  if ((s->tcmask & 1) && s->tx == 4) {
    CUtensorMap m;
    if (!make_map_2d_f32(&m, Y_dev, s->N / s->n[0] * blk, s->n[0], s->n[0], 32, 128)) {
      set_err(s, "slice address unusable for TMA (16-byte alignment)%s%lld", "", 0);
      return TUCKER_EINVAL;
    }
    static_assert(sizeof(m) == sizeof(sa.map), "descriptor size");
    memcpy(sa.map, &m, sizeof(m));
  }
  sa.y = Y_dev;
  CK(launch_set_slot(s->ctl, sa, st));
  return TUCKER_OK;
}

// Batches of tucker_stream_update_batched, one per set of states (in call order), captured with
// the slice read from each state's control block; a state's destruction drops every batch
// holding it.
std::mutex g_auto_mu;
std::vector<tucker_batch*> g_auto_batches;

tucker_status batch_create(tucker_state* const* states, const void* const* Y_slots_dev,
                           int32_t count, tucker_batch** out);

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

const char* tucker_version(void) { return kVersion; }

const char* tucker_last_error(const tucker_state* s) { return s ? s->err : "null state"; }

int64_t tucker_graph_kernels(const tucker_state* s) { return s ? s->graph_kernels : -1; }

int64_t tucker_block_graph_kernels(const tucker_state* s, int32_t nslices) {
  if (!s || nslices < 2 || nslices > 64) return -1;
  return s->bkernels[nslices];
}

tucker_status tucker_set_launch_plan(tucker_state* s, const tucker_launch_plan* p) {
  if (!s || !p) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  const int gp = p->grid_proj ? p->grid_proj : kGridP;
  const int gt = p->grid_tc ? p->grid_tc : s->nsm;
  const int gi = p->grid_isvd ? p->grid_isvd : kGridI;
  const int gc = p->grid_cv ? p->grid_cv : kGridCV;
  if (gp < 1 || gp > 4096 || gt < 1 || gt > s->nsm || gi < 1 || gi > kGridI || gc < 1 || gc > 65535) {
    set_err(s, "launch plan out of range%s%lld", "", 0);
    return TUCKER_EINVAL;
  }
  s->grid_p = gp;
  s->grid_tc = gt;
  s->grid_i = gi;
  s->grid_cv = gc;
  // the captured update graph holds the old launch shapes: capture again at the next update
  if (s->last_stream) cudaStreamSynchronize(s->last_stream);
  drop_graphs(s);
  return TUCKER_OK;
}

tucker_status tucker_get_launch_plan(const tucker_state* s, tucker_launch_plan* p) {
  if (!s || !p) return TUCKER_EINVAL;
  p->grid_proj = s->grid_p;
  p->grid_tc = s->grid_tc;
  p->grid_isvd = s->grid_i;
  p->grid_cv = s->grid_cv;
  return TUCKER_OK;
}

tucker_status tucker_init_sthosvd(const tucker_config* cfg, const void* X_dev, int64_t n_init,
                                  void* stream, tucker_state** out) {
  if (!out) return TUCKER_EINVAL;
  *out = nullptr;
  char msg[256];
  if (!validate(cfg, n_init, msg, sizeof(msg))) {
    fprintf(stderr, "tucker_init_sthosvd: %s\n", msg);
    return TUCKER_EINVAL;
  }
  if (!X_dev) return TUCKER_EINVAL;
  tucker_state* s = new tucker_state();
  s->cfg = *cfg;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  tucker_status rc = allocate(s, n_init);
  if (rc != TUCKER_OK) {
    if (rc == TUCKER_ECUDA) rc = TUCKER_ENOMEM;
    fprintf(stderr, "tucker_init_sthosvd: %s\n", s->err);
    free_all(s);
    delete s;
    return rc;
  }
  const bool mixed = cfg->precision == TUCKER_PREC_MIXED;
  const bool f32 = cfg->dtype == TUCKER_F32;
  if (mixed) rc = f32 ? do_init<float, float, float>(s, X_dev, n_init, st) : do_init<double, float, float>(s, X_dev, n_init, st);
  else rc = f32 ? do_init<float, double, double>(s, X_dev, n_init, st) : do_init<double, double, double>(s, X_dev, n_init, st);
  if (rc != TUCKER_OK) {
    fprintf(stderr, "tucker_init_sthosvd: %s\n", s->err);
    cudaDeviceSynchronize();
    free_all(s);
    delete s;
    return rc;
  }
  *out = s;
  return TUCKER_OK;
}

tucker_status tucker_stream_update(tucker_state* s, const void* Y_dev, void* stream) {
  if (!s || !Y_dev) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  tucker_status rp = push_replay(s, st);
  if (rp != TUCKER_OK) return rp;
  // Graph form (unless phase profiling is on): the update is captured once; each call writes
  // the slice's address (and its TMA descriptor) into the control block with a one-block kernel
  // and launches the graph.
  if (!s->prof && !s->graph_failed) {
    if (!s->uexec && capture_update(s, 1, &s->ugraph, &s->uexec, &s->graph_kernels) != TUCKER_OK)
      s->graph_failed = true;
    if (s->uexec) {
      tucker_status rs = write_slot(s, Y_dev, st);
      if (rs != TUCKER_OK) return rs;
      CK(cudaGraphLaunch(s->uexec, st));
      return TUCKER_OK;
    }
  }
  return update_dispatch(s, Y_dev, st);
}

tucker_status tucker_stream_update_block(tucker_state* s, const void* Y_dev, int32_t nslices,
                                         void* stream) {
  if (!s || !Y_dev || nslices < 1) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  if (nslices > s->block_cap) {
    set_err(s, "tucker_stream_update_block: %s%lld slices above the state's block_cap", "", nslices);
    return TUCKER_EINVAL;
  }
  if (nslices == 1) return tucker_stream_update(s, Y_dev, stream);
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  tucker_status rp = push_replay(s, st);
  if (rp != TUCKER_OK) return rp;
  // the spatial modes see the block as one tensor with a trailing mode of size nslices; graph
  // form (one graph per block size, captured at its first use) unless phase profiling is on
  const int b = nslices;
  if (!s->prof && !s->graph_failed) {
    if (!s->bexec[b] && capture_update(s, b, &s->bgraph[b], &s->bexec[b], &s->bkernels[b]) != TUCKER_OK)
      s->graph_failed = true;
    if (s->bexec[b]) {
      tucker_status rs = write_slot(s, Y_dev, st, b);
      if (rs != TUCKER_OK) return rs;
      CK(cudaGraphLaunch(s->bexec[b], st));
      return TUCKER_OK;
    }
  }
  s->blk = nslices;
  const tucker_status rc = update_dispatch(s, Y_dev, st);
  s->blk = 1;
  return rc;
}

tucker_status tucker_stream_update_host(tucker_state* s, const void* Y_host, void* stream) {
  if (!s || !Y_host) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = (size_t)s->N * (size_t)s->tx;
  if (!s->hcs) {
    // created into locals and committed to the state only when every step succeeded, so that a
    // failure leaves nothing half made (the next call starts over)
    void* stage[2] = {nullptr, nullptr};
    cudaStream_t cs = nullptr;
    cudaEvent_t cp[2] = {nullptr, nullptr}, cn[2] = {nullptr, nullptr};
    cudaError_t e = cudaSuccess;
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) e = cudaMalloc(&stage[b], bytes);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
      e = cudaEventCreateWithFlags(&cp[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&cn[b], cudaEventDisableTiming);
      if (e == cudaSuccess) e = cudaEventRecord(cn[b], st);   // both buffers free
    }
    if (e != cudaSuccess) {
      for (int b = 0; b < 2; ++b) {
        if (stage[b]) cudaFree(stage[b]);
        if (cp[b]) cudaEventDestroy(cp[b]);
        if (cn[b]) cudaEventDestroy(cn[b]);
      }
      if (cs) cudaStreamDestroy(cs);
      cudaGetLastError();
      set_err(s, "cannot set up the host-input staging buffers%s (%lld bytes each)", "", (long long)bytes);
      return e == cudaErrorMemoryAllocation ? TUCKER_ENOMEM : TUCKER_ECUDA;
    }
    for (int b = 0; b < 2; ++b) {
      s->hstage[b] = stage[b];
      s->allocs.push_back(stage[b]);
      s->hcopied[b] = cp[b];
      s->hconsumed[b] = cn[b];
    }
    s->hcs = cs;
  }
  const int b = s->hnext;
  s->hnext ^= 1;
  // the copy into buffer b waits for the update that last read it; the update waits for the copy
  CK(cudaStreamWaitEvent(s->hcs, s->hconsumed[b], 0));
  CK(cudaMemcpyAsync(s->hstage[b], Y_host, bytes, cudaMemcpyHostToDevice, s->hcs));
  CK(cudaEventRecord(s->hcopied[b], s->hcs));
  CK(cudaStreamWaitEvent(st, s->hcopied[b], 0));
  const tucker_status rc = tucker_stream_update(s, s->hstage[b], stream);
  if (rc != TUCKER_OK) return rc;
  CK(cudaEventRecord(s->hconsumed[b], st));
  return TUCKER_OK;
}

tucker_status tucker_reconstruct(tucker_state* s, int64_t t_begin, int64_t t_end, void* out_dev,
                                 void* stream) {
  if (!s || !out_dev) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  s->last_stream = (cudaStream_t)stream;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  if (t_begin < 0 || t_end > s->hctl->nd || t_begin >= t_end) {
    set_err(s, "slice range out of bounds%s (n_d = %lld)", "", s->hctl->nd);
    return TUCKER_EINVAL;
  }
  if (s->tw == 4) return do_reconstruct<float>(s, t_begin, t_end, out_dev, (cudaStream_t)stream);
  return do_reconstruct<double>(s, t_begin, t_end, out_dev, (cudaStream_t)stream);
}

tucker_status tucker_reconstruct_noalloc(tucker_state* s, int64_t t_begin, int64_t t_end,
                                         void* out_dev, void* stream) {
  if (!s || !out_dev) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  s->last_stream = (cudaStream_t)stream;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  if (t_begin < 0 || t_end > s->hctl->nd || t_begin >= t_end) {
    set_err(s, "slice range out of bounds%s (n_d = %lld)", "", s->hctl->nd);
    return TUCKER_EINVAL;
  }
  if (s->tw == 4) return do_reconstruct_noalloc<float>(s, t_begin, t_end, out_dev, (cudaStream_t)stream);
  return do_reconstruct_noalloc<double>(s, t_begin, t_end, out_dev, (cudaStream_t)stream);
}

tucker_status tucker_error_norm(tucker_state* s, double* err_bound, double* data_norm) {
  if (!s || !err_bound || !data_norm) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  *err_bound = std::sqrt(std::max(s->hctl->err2, 0.0));
  *data_norm = std::sqrt(std::max(s->hctl->data2, 0.0));
  return TUCKER_OK;
}

tucker_status tucker_error_norm_async(tucker_state* s, double* out2, void* stream) {
  if (!s || !out2) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  static_assert(offsetof(Ctl, data2) == offsetof(Ctl, err2) + sizeof(double), "err2, data2 adjacent");
  // Pinned (mapped) or managed destination: one GPU thread stores the two values over the host
  // link. A copy-engine read would queue behind host-to-device slice copies that other streams
  // have in flight, serializing a pipelined caller's copies with its updates.
  cudaPointerAttributes pa{};
  double* dptr = nullptr;
  if (cudaPointerGetAttributes(&pa, out2) == cudaSuccess) {
    if (pa.type == cudaMemoryTypeHost || pa.type == cudaMemoryTypeManaged)
      dptr = static_cast<double*>(pa.devicePointer);
  } else {
    cudaGetLastError();   // unregistered memory on older runtimes: use the copy
  }
  if (dptr) {
    CK(launch_read_err(s->ctl, dptr, (cudaStream_t)stream));
  } else {
    CK(cudaMemcpyAsync(out2, reinterpret_cast<unsigned char*>(s->ctl) + offsetof(Ctl, err2),
                       2 * sizeof(double), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
  }
  return TUCKER_OK;
}

tucker_status tucker_get_ranks(tucker_state* s, int64_t* ranks, int64_t* n_d) {
  if (!s || !ranks) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  for (int k = 0; k < s->d; ++k) ranks[k] = s->hctl->r[k];
  if (n_d) *n_d = s->hctl->nd;
  return TUCKER_OK;
}

tucker_status tucker_get_step_info(tucker_state* s, tucker_step_info* info) {
  if (!s || !info) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  memset(info, 0, sizeof(*info));
  info->eps = c.eps;
  info->y_norm2 = c.y2;
  double disc = 0.0;
  for (int k = 0; k < s->d - 1; ++k) {
    info->e_norm2[k] = c.e2[k];
    info->grew[k] = c.grew[k];
    info->r_add[k] = c.radd[k];
    disc += c.disc[k];
  }
  info->q = c.q;
  info->augmented = c.aug;
  info->r_stream = c.r[s->d - 1];
  info->discarded = disc + (c.aug ? 0.0 : c.q2) + c.dropped;
  return TUCKER_OK;
}

tucker_status tucker_get_step_log(tucker_state* s, int64_t first, int64_t count,
                                  tucker_step_record* out) {
  if (!s || !out || first < 0 || count < 0) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const long long have = std::min<long long>(s->hctl->nupdates, s->log_cap);
  if (first + count > have) {
    set_err(s, "step log holds updates [0, %s%lld)", "", have);
    return TUCKER_EINVAL;
  }
  if (count == 0) return TUCKER_OK;
  CK(cudaMemcpyAsync(out, s->log + first, sizeof(StepRec) * (size_t)count, cudaMemcpyDeviceToHost,
                     s->last_stream));
  CK(cudaStreamSynchronize(s->last_stream));
  return TUCKER_OK;
}

tucker_status tucker_replay_next(tucker_state* s, const tucker_replay* r) {
  if (!s || !r) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  for (int k = 0; k < s->d - 1; ++k) {
    if (r->grow[k] < -1 || r->grow[k] > s->n[k]) {
      set_err(s, "replay: grow[%s%lld] out of range", "", k);
      return TUCKER_EINVAL;
    }
  }
  if (r->augment < -1 || r->augment > 1) return TUCKER_EINVAL;
  if (!s->rp_host) CK(cudaMallocHost((void**)&s->rp_host, kReplayBytes));
  // the staging words of an earlier replay must have reached the device
  CK(cudaStreamSynchronize(s->last_stream));
  s->rp_host[0] = 1;
  for (int k = 0; k < TK_MAXD; ++k) s->rp_host[1 + k] = (k < s->d - 1) ? r->grow[k] : -1;
  s->rp_host[1 + TK_MAXD] = r->augment;
  s->rp_pending = true;
  return TUCKER_OK;
}

// ||G - I||_F of G = U^T U for a factor whose element (t, c) sits at U[t ut + c uc].
static tucker_status gram_dev(tucker_state* s, const double* U, long long ut, long long uc, int rows,
                              int r, double* G, double* part, double* out, cudaStream_t st) {
  CK(launch_gemm64(U, uc, ut, r, rows, U, ut, uc, r, G, 1, r, nullptr, st));
  CK(launch_frob_minus_i(G, r, part, 64, st));
  double hp[64];
  CK(cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  double a = 0.0;
  for (double v : hp) a += v;
  *out = std::sqrt(a);
  return TUCKER_OK;
}

tucker_status tucker_orthogonality_error(tucker_state* s, double* out) {
  if (!s || !out) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  const cudaStream_t st = s->last_stream;
  int rmax = 1;
  for (int k = 0; k < s->d; ++k) rmax = std::max(rmax, c.r[k]);
  double *G = nullptr, *part = nullptr;
  if (cudaMalloc(&G, sizeof(double) * (size_t)rmax * rmax) != cudaSuccess) return TUCKER_ENOMEM;
  if (cudaMalloc(&part, sizeof(double) * 64) != cudaSuccess) { cudaFree(G); return TUCKER_ENOMEM; }
  for (int k = 0; k < s->d && rc == TUCKER_OK; ++k) {
    if (k < s->d - 1) rc = gram_dev(s, s->U[k], 1, s->n[k], s->n[k], c.r[k], G, part, &out[k], st);
    else rc = gram_dev(s, s->Ud[c.ubuf], s->ldc, 1, c.nd, c.r[k], G, part, &out[k], st);
  }
  cudaFree(G);
  cudaFree(part);
  return rc;
}

tucker_status tucker_restore_orthogonality(tucker_state* s, void* stream, double* change) {
  if (!s) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  Ctl& h = *s->hctl;
  const int rd = h.r[s->d - 1], nd = h.nd, ld = s->ldc;
  double* Ud = s->Ud[h.ubuf];
  const size_t ubytes = sizeof(double) * (size_t)nd * ld;
  double *U0 = nullptr, *Un = nullptr, *G = nullptr, *T = nullptr, *part = nullptr;
  auto cleanup = [&]() { cudaFree(U0); cudaFree(Un); cudaFree(G); cudaFree(T); cudaFree(part); };
  if (cudaMalloc(&U0, ubytes) != cudaSuccess || cudaMalloc(&Un, ubytes) != cudaSuccess ||
      cudaMalloc(&G, sizeof(double) * rd * rd) != cudaSuccess ||
      cudaMalloc(&T, sizeof(double) * rd * rd) != cudaSuccess ||
      cudaMalloc(&part, sizeof(double) * 64) != cudaSuccess) {
    cleanup();
    return TUCKER_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(U0, Ud, ubytes, cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Un, Ud, ubytes, cudaMemcpyDeviceToDevice, st);
  // two Newton-Schulz steps U <- U (3 I - U^T U) / 2 towards the polar factor (quadratic once
  // ||U^T U - I|| < 1; the streaming factor's deviation is at rounding level)
  for (int pass = 0; pass < 2 && e == cudaSuccess; ++pass) {
    e = launch_gemm64(Ud, 1, ld, rd, nd, Ud, ld, 1, rd, G, 1, rd, nullptr, st);
    if (e == cudaSuccess) e = launch_ns_matrix(G, rd, T, st);
    if (e == cudaSuccess) e = launch_gemm64(Ud, ld, 1, nd, rd, T, 1, rd, rd, Un, ld, 1, nullptr, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(Ud, Un, ubytes, cudaMemcpyDeviceToDevice, st);
  }
  double hp[64];
  if (e == cudaSuccess) e = launch_change_norm(Ud, U0, nd, rd, ld, s->S, part, 64, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(hp, part, sizeof(hp), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cleanup();
    set_err(s, "tucker_restore_orthogonality: %s", cudaGetErrorString(e), 0);
    return TUCKER_ECUDA;
  }
  double c2 = 0.0;
  for (double v : hp) c2 += v;
  const double dchange = std::sqrt(c2);
  const double b = std::sqrt(std::max(h.err2, 0.0));
  h.err2 = (b + dchange) * (b + dchange);
  e = cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cleanup();
  if (e != cudaSuccess) CK(e);
  if (change) *change = dchange;
  return TUCKER_OK;
}

tucker_status tucker_test_stall_next(tucker_state* s) {
  if (!s) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  const int one = 1;
  CK(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(s->ctl) + offsetof(Ctl, test_stall), &one,
                     sizeof(int), cudaMemcpyHostToDevice, s->last_stream));
  CK(cudaStreamSynchronize(s->last_stream));
  return TUCKER_OK;
}

tucker_status tucker_recompress(tucker_state* s, double tau_total, void* stream,
                                tucker_recompress_info* info) {
  if (!s || !(tau_total > 0.0)) return TUCKER_EINVAL;
  if (!usable(s)) return TUCKER_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  s->last_stream = st;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const int d = s->d;
  Ctl c = *s->hctl;
  long long R = 1;
  for (int k = 0; k < d - 1; ++k) R *= c.r[k];
  const int rd = c.r[d - 1];
  const double b = std::sqrt(std::max(c.err2, 0.0));
  const double budget = tau_total * std::sqrt(c.data2) - b;
  if (!(budget > 0.0)) {
    set_err(s, "tucker_recompress: tau_total leaves no error budget beyond the running bound");
    return TUCKER_EINVAL;
  }
  // the core as the data of a batch ST-HOSVD (an FP64 state of sizes r_1 x ... x r_{d-1} with
  // r_d "slices"): its factors Q_k, core C', S', V' and discarded energy
  std::vector<void*> tmpbufs;
  auto dmalloc = [&](size_t bytes) -> void* {
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    tmpbufs.push_back(p);
    return p;
  };
  auto cleanup = [&]() { for (void* p : tmpbufs) cudaFree(p); };
  double* C64 = (double*)dmalloc(sizeof(double) * (size_t)R * rd);
  double* part = (double*)dmalloc(sizeof(double) * 1024);
  if (!C64 || !part) { cleanup(); return TUCKER_ENOMEM; }
  rc = tucker_copy_core(s, C64);
  if (rc != TUCKER_OK) { cleanup(); return rc; }
  std::vector<double> parts(1024);
  cudaError_t e = launch_norm2<double>(C64, R * rd, part, 1024, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(parts.data(), part, sizeof(double) * 1024, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) { cleanup(); CK(e); }
  double c2 = 0.0;
  for (double v : parts) c2 += v;
  tucker_config tc{};
  tc.ndim = d;
  tc.dtype = TUCKER_F64;
  tc.precision = TUCKER_PREC_FP64;
  for (int k = 0; k < d - 1; ++k) tc.n[k] = c.r[k];
  tc.rank_cap[d - 1] = rd;
  tc.steps_cap = rd + 1;
  tc.core_cap = R;
  tc.eps_m = s->cfg.eps_m;
  // eps' = tau' ||C|| / sqrt(d) = budget / sqrt(d) (||C|| = ||X^||, orthonormal factors)
  tc.tau = budget / std::sqrt(std::max(c2, 1e-300));
  tucker_state* t = nullptr;
  rc = tucker_init_sthosvd(&tc, C64, rd, stream, &t);
  if (rc != TUCKER_OK) { cleanup(); set_err(s, "tucker_recompress: ST-HOSVD of the core failed%s%lld", "", rc); return rc; }
  rc = sync_ctl(t);
  if (rc != TUCKER_OK) { tucker_destroy(t); cleanup(); return rc; }
  const Ctl ct = *t->hctl;
  long long Rn = 1;
  for (int k = 0; k < d - 1; ++k) Rn *= ct.r[k];
  const int rdn = ct.r[d - 1];
  double* Q = (double*)dmalloc(sizeof(double) * (size_t)TK_N_MAX * TK_N_MAX);
  double* Ck = (double*)dmalloc(sizeof(double) * (size_t)Rn * rdn);
  double* Vk = (double*)dmalloc(sizeof(double) * (size_t)Rn * rdn);
  const size_t un_elems = (size_t)std::max(TK_N_MAX, s->steps_cap) * TK_N_MAX;
  double* Un = (double*)dmalloc(sizeof(double) * un_elems);
  if (!Q || !Ck || !Vk || !Un) { tucker_destroy(t); cleanup(); return TUCKER_ENOMEM; }
  rc = tucker_copy_core(t, Ck);
  if (rc == TUCKER_OK) rc = tucker_copy_sv(t, s->S, Vk);
  // spatial factors U_k <- U_k Q_k (FP64 master and the work copy), streaming U_d <- U_d Q_d
  for (int k = 0; k < d && rc == TUCKER_OK; ++k) {
    rc = tucker_copy_factor(t, k, Q);   // r_k x r'_k, column-major
    if (rc != TUCKER_OK) break;
    if (k < d - 1) {
      // n_k x r'_k, column-major with leading dimension n_k (FP64 master, FP32 work copy)
      const int nk = s->n[k];
      float* uw = (s->tw == 4) ? static_cast<float*>(s->Uw[k]) : nullptr;
      e = launch_small_gemm(s->U[k], 1, nk, nk, c.r[k], Q, c.r[k], ct.r[k], Un, 1, nk, uw, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->U[k], Un, sizeof(double) * nk * ct.r[k], cudaMemcpyDeviceToDevice, st);
    } else {
      // n_d x r'_d rows of stride ldc; the columns past r'_d stay zero
      e = cudaMemsetAsync(Un, 0, sizeof(double) * (size_t)c.nd * s->ldc, st);
      if (e == cudaSuccess)
        e = launch_small_gemm(s->Ud[c.ubuf], s->ldc, 1, c.nd, rd, Q, rd, rdn, Un, s->ldc, 1, nullptr, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->Ud[c.ubuf], Un, sizeof(double) * (size_t)c.nd * s->ldc,
                            cudaMemcpyDeviceToDevice, st);
    }
    if (e != cudaSuccess) { rc = TUCKER_ECUDA; set_err(s, "tucker_recompress: %s", cudaGetErrorString(e), k); }
  }
  if (rc == TUCKER_OK) {
    const int ls = tk_cv_stride(rdn, s->ldc, s->tw);
    e = (s->tw == 4) ? launch_set_cv<float>(Ck, Vk, Rn, rdn, s->Cb[c.cbuf], s->Vb[c.cbuf], ls, st)
                     : launch_set_cv<double>(Ck, Vk, Rn, rdn, s->Cb[c.cbuf], s->Vb[c.cbuf], ls, st);
    if (e != cudaSuccess) { rc = TUCKER_ECUDA; set_err(s, "tucker_recompress: %s", cudaGetErrorString(e), 0); }
  }
  const double disc = std::max(ct.err2, 0.0);
  tucker_destroy(t);
  if (rc == TUCKER_OK) {
    Ctl& h = *s->hctl;
    for (int k = 0; k < d; ++k) { h.r[k] = ct.r[k]; h.rold[k] = ct.r[k]; }
    h.err2 = (b + std::sqrt(disc)) * (b + std::sqrt(disc));
    h.xbuf = -1;
    e = cudaMemcpyAsync(s->ctl, &h, sizeof(Ctl), cudaMemcpyHostToDevice, st);
    // TF32 hi/lo splits of the new spatial factors for the tensor-core passes (they read the
    // ranks from the control block just written)
    for (int k = 0; k < d - 1 && e == cudaSuccess; ++k)
      if ((s->tcmask >> k) & 1) e = split_u(s, k, 0, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { rc = TUCKER_ECUDA; set_err(s, "tucker_recompress: %s", cudaGetErrorString(e), 0); }
  }
  cleanup();
  if (rc == TUCKER_OK && info) {
    info->discarded = disc;
    info->err_bound = b + std::sqrt(disc);
    for (int k = 0; k < TUCKER_MAX_MODES; ++k) info->ranks[k] = k < d ? ct.r[k] : 0;
  }
  return rc;
}

tucker_status tucker_copy_factor(tucker_state* s, int32_t mode, double* dst) {
  if (!s || !dst || mode < 0 || mode >= s->d) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  if (mode < s->d - 1) {
    CK(cudaMemcpyAsync(dst, s->U[mode], sizeof(double) * s->n[mode] * c.r[mode],
                       cudaMemcpyDeviceToDevice, s->last_stream));
  } else {
    CK(launch_ud_to_colmajor(s->Ud[c.ubuf], c.nd, c.r[s->d - 1], s->ldc, dst, s->last_stream));
  }
  CK(cudaStreamSynchronize(s->last_stream));
  return TUCKER_OK;
}

tucker_status tucker_copy_core(tucker_state* s, double* dst) {
  if (!s || !dst) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  long long R = 1;
  for (int i = 0; i < s->d - 1; ++i) R *= c.r[i];
  const int ls = tk_cv_stride(c.r[s->d - 1], s->ldc, s->tw);
  if (s->tw == 4) CK(launch_state_to_colmajor<float>(s->Cb[c.cbuf], R, c.r[s->d - 1], ls, dst, s->last_stream));
  else CK(launch_state_to_colmajor<double>(s->Cb[c.cbuf], R, c.r[s->d - 1], ls, dst, s->last_stream));
  CK(cudaStreamSynchronize(s->last_stream));
  return TUCKER_OK;
}

tucker_status tucker_copy_sv(tucker_state* s, double* S_dev, double* V_dev) {
  if (!s) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  const Ctl& c = *s->hctl;
  const int rd = c.r[s->d - 1];
  if (S_dev) CK(cudaMemcpyAsync(S_dev, s->S, sizeof(double) * rd, cudaMemcpyDeviceToDevice, s->last_stream));
  if (V_dev) {
    long long R = 1;
    for (int i = 0; i < s->d - 1; ++i) R *= c.r[i];
    const int ls = tk_cv_stride(rd, s->ldc, s->tw);
    if (s->tw == 4) CK(launch_state_to_colmajor<float>(s->Vb[c.cbuf], R, rd, ls, V_dev, s->last_stream));
    else CK(launch_state_to_colmajor<double>(s->Vb[c.cbuf], R, rd, ls, V_dev, s->last_stream));
  }
  CK(cudaStreamSynchronize(s->last_stream));
  return TUCKER_OK;
}

tucker_status tucker_batch_create(tucker_state* const* states, const void* const* Y_slots_dev,
                                  int32_t count, tucker_batch** out) {
  if (!Y_slots_dev || count < 1) return TUCKER_EINVAL;
  for (int i = 0; i < count; ++i)
    if (!Y_slots_dev[i]) return TUCKER_EINVAL;
  return batch_create(states, Y_slots_dev, count, out);
}

}  // extern "C"

namespace {
// tucker_batch_create without the slot check: a NULL slot makes that state's branch read its slice
// from the state's control block (tucker_stream_update_batched writes it before each launch).
tucker_status batch_create(tucker_state* const* states, const void* const* Y_slots_dev,
                           int32_t count, tucker_batch** out) {
  if (!out) return TUCKER_EINVAL;
  *out = nullptr;
  if (!states || !Y_slots_dev || count < 1 || count > 4096) return TUCKER_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!states[i]) return TUCKER_EINVAL;
    if (!usable(states[i])) return TUCKER_ESTATE;
    for (int j = 0; j < i; ++j)
      if (states[j] == states[i]) return TUCKER_EINVAL;   // a state updates once per launch
  }
  tucker_batch* b = new tucker_batch();
  b->states.assign(states, states + count);
  std::vector<cudaStream_t> streams(count + 1, nullptr);
  std::vector<cudaEvent_t> evs(count + 1, nullptr);
  tucker_status rc = TUCKER_OK;
  for (int i = 0; i <= count && rc == TUCKER_OK; ++i) {
    if (cudaStreamCreateWithFlags(&streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&evs[i], cudaEventDisableTiming) != cudaSuccess) rc = TUCKER_ECUDA;
  }
  // the states' earlier work must be complete before the graph is first launched; the capture
  // itself enqueues nothing
  for (int i = 0; i < count && rc == TUCKER_OK; ++i)
    if (cudaStreamSynchronize(states[i]->last_stream) != cudaSuccess) rc = TUCKER_ECUDA;
  if (rc == TUCKER_OK) rc = capture_batch(b, Y_slots_dev, streams.data(), evs.data());
  for (int i = 0; i <= count; ++i) {
    if (streams[i]) cudaStreamDestroy(streams[i]);
    if (evs[i]) cudaEventDestroy(evs[i]);
  }
  if (rc != TUCKER_OK) {
    fprintf(stderr, "tucker_batch_create: %s\n", b->err);
    tucker_batch_destroy(b);
    return rc;
  }
  *out = b;
  return TUCKER_OK;
}
}  // namespace

extern "C" {

tucker_status tucker_batch_update(tucker_batch* b, void* stream) {
  if (!b || !b->exec) return TUCKER_EINVAL;
  for (tucker_state* s : b->states)
    if (!usable(s)) return TUCKER_ESTATE;
  cudaStream_t st = (cudaStream_t)stream;
  for (tucker_state* s : b->states)
    if (push_replay(s, st) != TUCKER_OK) return TUCKER_ECUDA;
  if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return TUCKER_ECUDA;
  for (tucker_state* s : b->states) s->last_stream = st;
  return TUCKER_OK;
}

int64_t tucker_batch_kernels(const tucker_batch* b) { return b ? b->launches : -1; }

tucker_status tucker_stream_update_batched(tucker_state* const* states, const void* const* Y_dev,
                                           int32_t count, void* stream) {
  if (!states || !Y_dev || count < 1 || count > 4096) return TUCKER_EINVAL;
  for (int i = 0; i < count; ++i) {
    if (!states[i] || !Y_dev[i]) return TUCKER_EINVAL;
    if (!usable(states[i])) return TUCKER_ESTATE;
  }
  std::lock_guard<std::mutex> lock(g_auto_mu);
  tucker_batch* b = nullptr;
  for (tucker_batch* c : g_auto_batches)
    if ((int)c->states.size() == count && std::equal(c->states.begin(), c->states.end(), states)) b = c;
  if (!b) {
    // first call for this set of states: one graph, each branch reading its state's slice from
    // the control block (written below by the slot kernels)
    std::vector<const void*> none(count, nullptr);
    tucker_status rc = batch_create(states, none.data(), count, &b);
    if (rc != TUCKER_OK) return rc;
    g_auto_batches.push_back(b);
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int i = 0; i < count; ++i) {
    tucker_status rc = write_slot(states[i], Y_dev[i], st);
    if (rc != TUCKER_OK) return rc;
  }
  return tucker_batch_update(b, stream);
}

void tucker_batch_destroy(tucker_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  delete b;
}

tucker_status tucker_profile_enable(tucker_state* s, int32_t on) {
  if (!s) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  s->prof = on != 0;
  s->ev_used = 0;
  s->ev_phase.clear();
  s->prof_launches = 0;
  s->prof_updates = 0;
  for (int i = 0; i < TK_NPH; ++i) s->bytes0[i] = s->hctl->acc_bytes[i];
  return TUCKER_OK;
}

tucker_status tucker_profile_read(tucker_state* s, tucker_profile* out) {
  if (!s || !out) return TUCKER_EINVAL;
  tucker_status rc = sync_ctl(s);
  if (rc != TUCKER_OK) return rc;
  memset(out, 0, sizeof(*out));
  for (size_t i = 0; i < s->ev_phase.size(); ++i) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, s->ev[2 * i], s->ev[2 * i + 1]));
    if (s->ev_phase[i] == TK_PH_SLICE) out->ms_slice_pass += ms;
    else out->ms[s->ev_phase[i]] += ms;
  }
  for (int i = 0; i < TK_NPH; ++i) out->bytes[i] = s->hctl->acc_bytes[i] - s->bytes0[i];
  out->launches = s->prof_launches;
  out->updates = s->prof_updates;
  return TUCKER_OK;
}

void tucker_destroy(tucker_state* s) {
  if (!s) return;
  {
    // batches of tucker_stream_update_batched that hold this state go with it
    std::lock_guard<std::mutex> lock(g_auto_mu);
    for (size_t i = 0; i < g_auto_batches.size();) {
      tucker_batch* b = g_auto_batches[i];
      if (std::find(b->states.begin(), b->states.end(), s) != b->states.end()) {
        tucker_batch_destroy(b);
        g_auto_batches.erase(g_auto_batches.begin() + i);
      } else {
        ++i;
      }
    }
  }
  cudaStreamSynchronize(s->last_stream);
  if (s->hcs) {
    cudaStreamSynchronize(s->hcs);
    cudaStreamDestroy(s->hcs);
    for (int b = 0; b < 2; ++b) {
      cudaEventDestroy(s->hcopied[b]);
      cudaEventDestroy(s->hconsumed[b]);
    }
  }
  drop_graphs(s);
  if (s->cap_st) cudaStreamDestroy(s->cap_st);
  if (s->body_st) cudaStreamDestroy(s->body_st);
  free_all(s);
  delete s;
}

}  // extern "C"
