// Host runtime and C ABI (include/ccd.h): context, device scratch, launch
// sequence of Algorithm 1 (boxes, broad phase, narrow phase), status.

#include <algorithm>
#include <climits>
#include <utility>
#include <vector>
#include <cstdio>
#include <cstring>
#include <new>

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

using namespace ccd;

struct ccd_ctx {
  int device = 0;
  ccd_opts opts{};
  int sm_count = 0;
  int narrow_blocks = 0;
  DevCtl *ctl = nullptr;
  // broad-phase scratch, sized for cap_boxes boxes
  int64_t cap_boxes = 0;
  void *broad_mem = nullptr;
  BroadBufs bb{};
  // pair buffer of ccd_step / ccd_step_batch: pair_cap pairs, vertex-face
  // from the front, edge-edge from the back (vf and ee point at the same
  // buffer)
  int64_t pair_cap = 0;
  int32_t *vf = nullptr, *ee = nullptr;
  // single-precision candidates of the strip sweep
  int64_t sup_cap = 0;
  uint2 *sup = nullptr;
  // narrow-phase scratch, sized for cap_q queries
  int64_t cap_q = 0;
  uint32_t *qflags = nullptr;
  unsigned long long *qiters = nullptr;
  unsigned long long *qrec = nullptr;          // query records, 24 x cap_q words
  int *qsid = nullptr;                         // scene of each query (batched scenes)
  double *prims = nullptr;                     // per-primitive set-up records of the narrow phase
  int64_t cap_prims = 0;                       // (words)
  // side stream of ccd_step: the per-primitive set-up runs beside the broad phase
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // batched scenes
  int64_t cap_bsid = 0, cap_scenes = 0;
  int *bsid = nullptr, *saxis = nullptr;
  float *ssum = nullptr;
  uint32_t *smm = nullptr;
  const unsigned long long *s_key_last = nullptr;   // sorted copy keys of the last broad phase
  SortWork sortw{};                                  // radix sort counters and look-back states
  int64_t last_ranges = 0;                          // ranges of the last memory-limited step
  // FP64 strip sweep buffers, sized for cap_boxes boxes (allocated on first use)
  int64_t cap_strips64 = 0;
  void *strips64_mem = nullptr;
  uint32_t *c_box = nullptr, *c_seg = nullptr, *s_seg = nullptr;
  long long *s_key64 = nullptr, *s_ahi64c = nullptr;
  longlong2 *s_oth64c = nullptr;
  StripParam *sparam_sc = nullptr;             // strip layout per scene (batched scenes)
  RingCell *ring = nullptr;
  unsigned long long ring_cap = 0;
  cudaStream_t last_stream = nullptr;
  int64_t last_nB = 0;
  long long n_launches = 0;
  // CUDA graphs of ccd_step (device output) and ccd_step_batch, captured on a
  // private stream and replayed on the caller's stream while the call's
  // arguments stay the same
  cudaStream_t cap_stream = nullptr;
  bool capturing = false;
  struct GraphEntry {
    bool valid = false;
    unsigned char key[256];
    cudaGraphExec_t exec = nullptr;
    long long launches = 0;
  } g_step, g_batch;
  // stage events: ev[2k] before stage k, ev[2k+1] after; ran[k] for the last call
  cudaEvent_t ev[2 * CCD_NSTAGES] = {};
  bool ran[CCD_NSTAGES] = {};
};

namespace {

#define CK(call)                                                     \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) {                                         \
      std::fprintf(stderr, "ccd: %s failed: %s\n", #call, cudaGetErrorString(e_)); \
      return e_ == cudaErrorMemoryAllocation ? CCD_ENOMEM : CCD_ECUDA; \
    }                                                                \
  } while (0)

inline int64_t cdiv(int64_t a, int64_t b) { return (a + b - 1) / b; }

inline void mark(ccd_ctx *c, int stage, bool begin, cudaStream_t s) {
  if (!c->opts.profile_stages || c->capturing) return;
  cudaEventRecord(c->ev[2 * stage + (begin ? 0 : 1)], s);
  if (!begin) c->ran[stage] = true;
}
inline void clear_marks(ccd_ctx *c) {
  for (int k = 0; k < CCD_NSTAGES; ++k) c->ran[k] = false;
}

__global__ void k_reset_broad(DevCtl *c) {
  c->n_vf = c->n_ee = c->n_superset = 0;
  c->n_copies = 0;
  c->strip_fallback = 0;
  c->sup_overflow = 0;
  c->copy_oversize = 0;
  for (int i = 0; i < 6; ++i) c->var_sum[i] = 0;
  c->axis = 0;
}
// keep_toi: a later batch of the same step (the earliest time carries over)
__global__ void k_reset_narrow(DevCtl *c, int keep_toi) {
  c->q_next = 0;
  c->pending = 0;
  if (!keep_toi) c->toi_bits = 0x7FF0000000000000ull;
  c->n_intervals = c->n_exported = c->n_capped = c->queue_peak = 0;
  c->t_start = c->t_exhausted = c->t_end = 0;
  c->n_donated = 0;
  c->n_intervals_tail = 0;
  c->n_intervals_fp64 = 0;
  c->n_left = 0;
}
__global__ void k_reset_status(DevCtl *c) { c->status = CCD_OK; }
__global__ void k_add_pending(DevCtl *c, unsigned long long n) { c->pending += n; }

// Pair counts of the broad phase clamped to the buffer capacities (ccd_step:
// the narrow phase reads them on the device, no host round trip).
// Pair counts of the shared pair buffer (cap pairs, vertex-face from the
// front, edge-edge from the back), clamped so that the two lists do not
// overlap; pairs that did not fit raise CCD_ETRUNC (the first error wins).
__global__ void k_counts_from_broad(DevCtl *c, int64_t cap) {
  const unsigned long long a = c->n_vf, b = c->n_ee, uc = (unsigned long long)cap;
  const unsigned long long va = min(a, uc);
  c->pair_counts[0] = (long long)va;
  c->pair_counts[1] = (long long)min(b, uc - va);
  if (a + b > uc || c->sup_overflow) atomicCAS(&c->status, CCD_OK, CCD_ETRUNC);
}

int ensure_broad(ccd_ctx *c, int64_t nB) {
  if (nB <= c->cap_boxes) return CCD_OK;
  if (c->broad_mem) CK(cudaFree(c->broad_mem));
  c->broad_mem = nullptr;
  c->cap_boxes = 0;
  int64_t cap = std::max<int64_t>(nB, 1024);
  // box copies of the strip sweep: a box lands in at most (its width / the
  // strip width) + 2 strips, +1 for rounding, so strips two mean widths wide
  // bound the total by 3.5 nB (typically about 1.5 nB); the buffers hold
  // 3 nB + 4096 copies, and past that the device falls back to one strip per
  // scene (the plain sweep)
  const int64_t capc = 3 * cap + 4096;
  int64_t nbuild = cdiv(cap, kBuildThreads);
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t off = bytes; bytes += (n + 255) & ~size_t(255); return off; };
  size_t o_lo32 = take(3 * cap * sizeof(float)), o_hi32 = take(3 * cap * sizeof(float));
  size_t o_lo64 = take(3 * cap * sizeof(long long)), o_hi64 = take(3 * cap * sizeof(long long));
  size_t o_vid = take(cap * sizeof(int4));
  size_t o_k0 = take(capc * 8), o_k1 = take(capc * 8), o_v0 = take(capc * 4), o_v1 = take(capc * 4);
  size_t o_sortw = take(sort_work_bytes(capc));
  size_t o_salo = take(cap * 4), o_sahi = take(capc * 4);
  size_t o_soth = take(capc * sizeof(float4)), o_svid = take(capc * sizeof(int4)), o_stag = take(capc);
  size_t o_part = take(kStatWords * nbuild * sizeof(float));
  size_t o_salo64 = take(cap * 8), o_sahi64 = take(cap * 8), o_soth64 = take(2 * cap * sizeof(longlong2));
  size_t o_clocal = take(cap * 4), o_cblk = take((cdiv(cap, kCopyBlock) + 1) * 8);
  size_t o_sp1 = take(sizeof(StripParam));
  char *m = nullptr;
  CK(cudaMalloc(&m, bytes));
  c->broad_mem = m;
  c->cap_boxes = cap;
  BroadBufs &B = c->bb;
  B.lo32 = (float *)(m + o_lo32);
  B.hi32 = (float *)(m + o_hi32);
  B.lo64 = (long long *)(m + o_lo64);
  B.hi64 = (long long *)(m + o_hi64);
  B.vid = (int4 *)(m + o_vid);
  B.keys[0] = m + o_k0;
  B.keys[1] = m + o_k1;
  B.vals[0] = (uint32_t *)(m + o_v0);
  B.vals[1] = (uint32_t *)(m + o_v1);
  CK(cudaMemset(m + o_sortw, 0, sort_work_bytes(capc)));   // the sort's counters start at zero
  c->sortw = sort_work_at(m + o_sortw);
  B.s_alo = (float *)(m + o_salo);
  B.s_ahi = (float *)(m + o_sahi);
  B.s_oth = (float4 *)(m + o_soth);
  B.s_vid = (int4 *)(m + o_svid);
  B.s_tag = (uint8_t *)(m + o_stag);
  B.partials = (float *)(m + o_part);
  B.s_alo64 = (long long *)(m + o_salo64);
  B.s_ahi64 = (long long *)(m + o_sahi64);
  B.s_oth64 = (longlong2 *)(m + o_soth64);
  B.cap_copies = capc;
  B.c_local = (uint32_t *)(m + o_clocal);
  B.c_blk = (unsigned long long *)(m + o_cblk);
  B.sparam = (StripParam *)(m + o_sp1);
  return CCD_OK;
}

int ensure_narrow(ccd_ctx *c, int64_t nq, cudaStream_t s) {
  if (!c->ring) {
    unsigned long long cap = c->opts.queue_capacity > 0 ? (unsigned long long)c->opts.queue_capacity : (1ull << 21);
    if (cap & (cap - 1)) return CCD_EINVAL;
    CK(cudaMalloc(&c->ring, cap * sizeof(RingCell)));
    c->ring_cap = cap;
    // ring positions start at 0: cell i expects sequence number i
    k_ring_init<<<(unsigned)std::min<unsigned long long>(cdiv(cap, 256), 4096), 256, 0, s>>>(c->ring, cap, 0);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(&c->ctl->q_head, 0, sizeof(unsigned long long), s));
    CK(cudaMemsetAsync(&c->ctl->q_tail, 0, sizeof(unsigned long long), s));
  }
  if (nq <= c->cap_q) return CCD_OK;
  if (c->qflags) CK(cudaFree(c->qflags));
  if (c->qiters) CK(cudaFree(c->qiters));
  if (c->qrec) CK(cudaFree(c->qrec));
  if (c->qsid) CK(cudaFree(c->qsid));
  c->qflags = nullptr;
  c->qiters = nullptr;
  c->qrec = nullptr;
  c->qsid = nullptr;
  c->cap_q = 0;
  // a multiple of the narrow kernel's staged batch (and of 32): its record
  // copies stay aligned and in bounds
  constexpr int64_t kCapUnit = 32 * kStageQ;
  int64_t cap = (std::max<int64_t>(nq, 1024) + kCapUnit - 1) / kCapUnit * kCapUnit;
  CK(cudaMalloc(&c->qflags, cap * sizeof(uint32_t)));
  CK(cudaMalloc(&c->qiters, cap * sizeof(unsigned long long)));
  CK(cudaMalloc(&c->qrec, cap * (24 * sizeof(unsigned long long) + 33 * sizeof(float))));
  CK(cudaMalloc(&c->qsid, cap * sizeof(int)));
  c->cap_q = cap;
  return CCD_OK;
}

// Per-primitive set-up records of the narrow phase for a mesh of nV, nE, nF.
int ensure_prims(ccd_ctx *c, int64_t nV, int64_t nE, int64_t nF) {
  const int64_t pw = narrow_prim_words(nV, nE, nF);
  if (pw <= c->cap_prims) return CCD_OK;
  if (c->prims) CK(cudaFree(c->prims));
  c->prims = nullptr;
  c->cap_prims = 0;
  CK(cudaMalloc(&c->prims, pw * sizeof(double)));
  c->cap_prims = pw;
  return CCD_OK;
}

int ensure_strips64(ccd_ctx *c) {
  const int64_t capc = c->bb.cap_copies;
  if (capc <= c->cap_strips64) return CCD_OK;
  if (c->strips64_mem) CK(cudaFree(c->strips64_mem));
  c->strips64_mem = nullptr;
  c->cap_strips64 = 0;
  size_t bytes = 0;
  auto take = [&](size_t n) { size_t off = bytes; bytes += (n + 255) & ~size_t(255); return off; };
  const size_t o_box = take(capc * 4), o_seg = take(capc * 4), o_sseg = take(capc * 4);
  const size_t o_key = take(capc * 8), o_ahi = take(capc * 8), o_oth = take(2 * capc * sizeof(longlong2));
  char *m = nullptr;
  CK(cudaMalloc(&m, bytes));
  c->strips64_mem = m;
  c->c_box = (uint32_t *)(m + o_box);
  c->c_seg = (uint32_t *)(m + o_seg);
  c->s_seg = (uint32_t *)(m + o_sseg);
  c->s_key64 = (long long *)(m + o_key);
  c->s_ahi64c = (long long *)(m + o_ahi);
  c->s_oth64c = (longlong2 *)(m + o_oth);
  c->cap_strips64 = capc;
  return CCD_OK;
}

int ensure_scenes(ccd_ctx *c, int64_t nB, int64_t n_scenes) {
  if (nB > c->cap_bsid) {
    if (c->bsid) CK(cudaFree(c->bsid));
    c->bsid = nullptr;
    c->cap_bsid = 0;
    CK(cudaMalloc(&c->bsid, std::max<int64_t>(nB, 1024) * sizeof(int)));
    c->cap_bsid = std::max<int64_t>(nB, 1024);
  }
  if (n_scenes > c->cap_scenes) {
    if (c->ssum) CK(cudaFree(c->ssum));
    if (c->saxis) CK(cudaFree(c->saxis));
    if (c->smm) CK(cudaFree(c->smm));
    if (c->sparam_sc) CK(cudaFree(c->sparam_sc));
    c->ssum = nullptr;
    c->saxis = nullptr;
    c->smm = nullptr;
    c->sparam_sc = nullptr;
    c->cap_scenes = 0;
    CK(cudaMalloc(&c->ssum, 9 * n_scenes * sizeof(float)));
    CK(cudaMalloc(&c->saxis, n_scenes * sizeof(int)));
    CK(cudaMalloc(&c->smm, 6 * n_scenes * sizeof(uint32_t)));
    CK(cudaMalloc(&c->sparam_sc, n_scenes * sizeof(StripParam)));
    c->cap_scenes = n_scenes;
  }
  return CCD_OK;
}

int ensure_sup(ccd_ctx *c, int64_t cap) {
  cap = std::max<int64_t>(cap, 1 << 20);
  if (cap <= c->sup_cap) return CCD_OK;
  if (c->sup) CK(cudaFree(c->sup));
  c->sup = nullptr;
  c->sup_cap = 0;
  CK(cudaMalloc(&c->sup, cap * sizeof(uint2)));
  c->sup_cap = cap;
  return CCD_OK;
}

int ensure_pairs(ccd_ctx *c, int64_t cap) {
  int rc = ensure_sup(c, 2 * cap);
  if (rc) return rc;
  if (cap <= c->pair_cap) return CCD_OK;
  if (c->vf) CK(cudaFree(c->vf));
  c->vf = c->ee = nullptr;
  c->pair_cap = 0;
  CK(cudaMalloc(&c->vf, cap * 2 * sizeof(int32_t)));
  c->ee = c->vf;
  c->pair_cap = cap;
  return CCD_OK;
}

// Default pair capacity of ccd_step / ccd_step_batch: 4 pairs per box (the
// 512 x 512 folded cloth, a dense self-contact case, needs 3.2), at least
// 2^20; synchronous calls grow it on demand.
int64_t default_pair_capacity(int64_t nB) { return std::max<int64_t>(1 << 20, 4 * nB); }

bool mesh_args_ok(const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                  const int32_t *F, int64_t nF) {
  if (nV < 0 || nE < 0 || nF < 0) return false;
  if (nV + nE + nF >= (1ll << 31)) return false;
  if (nV > 0 && (!V0 || !V1)) return false;
  if ((nE > 0 && !E) || (nF > 0 && !F)) return false;
  return true;
}

// Launch sequence of the broad phase.  Outputs go to vf_out/ee_out (counts in
// ctl->n_vf / n_ee, unclamped).
struct SceneSpec {
  int n;                            // number of scenes (0: one scene, no offsets)
  const int64_t *voff, *eoff, *foff;
};

int launch_broad(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                 const int32_t *F, int64_t nF, int32_t *vf_out, int64_t vf_cap, int32_t *ee_out, int64_t ee_cap,
                 cudaStream_t s, const SceneSpec &sc = SceneSpec{0, nullptr, nullptr, nullptr}, bool ee_rev = false,
                 int phase = 3, int64_t i_begin = 0, int64_t i_end = INT64_MAX) {
  // phase 1: boxes and sort; phase 2: the sweep (over sorted copies
  // [i_begin, i_end) for the cell sweeps); 3: both
  const int64_t nB = nV + nE + nF;
  int rc = ensure_broad(c, nB);
  if (rc) return rc;
  if (!c->capturing) {
    rc = ensure_sup(c, ee_rev ? 2 * vf_cap : std::max<int64_t>(vf_cap + ee_cap, 8 * nB));
    if (rc) return rc;
  }
  if (sc.n > 0) {
    rc = ensure_scenes(c, nB, sc.n);
    if (rc) return rc;
  }
  c->last_nB = nB;
  if (phase & 1)
    k_reset_broad<<<1, 1, 0, s>>>(c->ctl);
  else
    k_reset_sweep<<<1, 1, 0, s>>>(c->ctl);
  if (nB == 0) {
    c->n_launches += 1;
    return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ECUDA;
  }
  BroadBufs B = c->bb;
  B.n_scenes = sc.n;
  B.voff = sc.voff;
  B.eoff = sc.eoff;
  B.foff = sc.foff;
  B.bsid = c->bsid;
  B.ssum = c->ssum;
  B.smm = c->smm;
  B.saxis = c->saxis;
  if (sc.n > 0) B.sparam = c->sparam_sc;
  B.strip_factor = c->opts.strip_width > 0 ? (float)c->opts.strip_width : 3.0f;
  const bool fp64 = c->opts.broad_fp64 != 0;
  // sweep: 0 cells, 1 warp per box, 2 tiled over one sorted list (the FP64
  // form has strips and warp per box; more than 65,536 scenes take the tiled
  // sweep: the strip keys hold 16 bits of scene index)
  int sweep = c->opts.sweep_kernel;
  if (fp64 && sweep == 2) sweep = 1;
  if (!fp64 && sweep == 0 && sc.n > 65536) sweep = 2;
  if (sweep == 0 && nB >= (1ll << 30)) sweep = fp64 ? 1 : 2;   // copies carry 2 flag bits above the box id
  const bool strips64 = fp64 && sweep == 0;
  B.strips_fp64 = strips64 ? 1 : 0;
  if (strips64 && !c->capturing) {
    rc = ensure_strips64(c);
    if (rc) return rc;
  }
  B.c_box = c->c_box;
  B.c_seg = c->c_seg;
  B.s_seg = c->s_seg;
  B.s_key64 = c->s_key64;
  B.s_ahi64c = c->s_ahi64c;
  B.s_oth64c = c->s_oth64c;
  const int nbuild = (int)cdiv(nB, kBuildThreads);
  const int grid = (int)std::min<int64_t>(cdiv(nB, 256), (int64_t)c->sm_count * 8);
  int sort_passes = 0;             // radix passes (one kernel each) ...
  int n_sorts = 0;                 // ... of this many sorts (one counting kernel each)
  int extra = 0;
  int sbits = 0;   // bits of the scene index in the keys of batched scenes
  while ((1ll << sbits) < sc.n) ++sbits;
  const unsigned long long *s_key = c->s_key_last;
  if (phase & 1) {
  sort_passes = fp64 ? 8 : 4;
  n_sorts = 1;
  mark(c, CCD_STAGE_BOXES, true, s);
  if (sc.n > 0) {
    CK(cudaMemsetAsync(c->ssum, 0, 9 * sc.n * sizeof(float), s));
    CK(cudaMemsetAsync(c->smm, 0xFF, 3 * sc.n * sizeof(uint32_t), s));
    CK(cudaMemsetAsync(c->smm + 3 * sc.n, 0, 3 * sc.n * sizeof(uint32_t), s));
    k_build_boxes<<<nbuild, kBuildThreads, 0, s>>>(nV, nE, nF, V0, V1, E, F, B);
    k_axis_select_scenes<<<(unsigned)cdiv(sc.n, 256), 256, 0, s>>>(B);
  } else {
    k_build_boxes<<<nbuild, kBuildThreads, 0, s>>>(nV, nE, nF, V0, V1, E, F, B);
    k_axis_select<<<1, 1024, 0, s>>>(B.partials, nbuild, nB, c->ctl, B.sparam, B.strip_factor);
  }
  mark(c, CCD_STAGE_BOXES, false, s);
  mark(c, CCD_STAGE_SORT, true, s);
  if (strips64) {
    // FP64 strips: copies sorted by the ordered FP64 minimum (64 bits), then
    // stably by strip segment (16 bits)
    const int nblk = (int)cdiv(nB, kCopyBlock);
    k_count_copies<<<nblk, kCopyBlock, 0, s>>>(nB, B, c->ctl);
    k_scan_copies<<<1, 1024, 0, s>>>(nblk, nB, B, c->ctl);
    k_expand_copies64<<<grid, 256, 0, s>>>(nB, B, c->ctl, (unsigned long long *)B.keys[0], B.vals[0]);
    const int cur = radix_sort(B.keys, B.vals, 8, B.cap_copies, c->sortw, s, &c->ctl->status, 64, &c->ctl->n_copies);
    const int cgrid = (int)std::min<int64_t>(cdiv(B.cap_copies, 256), (int64_t)c->sm_count * 8);
    uint32_t *ka = (uint32_t *)B.keys[cur ^ 1];
    void *k2[2] = {ka, ka + B.cap_copies};
    uint32_t *v2[2] = {B.vals[cur], B.vals[cur ^ 1]};
    k_gather_seg<<<cgrid, 256, 0, s>>>(B.cap_copies, c->ctl, B.vals[cur], B.c_seg, ka);
    const int cur2 = radix_sort(k2, v2, 4, B.cap_copies, c->sortw, s, &c->ctl->status, 24, &c->ctl->n_copies);
    k_gather_copies64<<<cgrid, 256, 0, s>>>(nB, B, c->ctl, v2[cur2]);
    sort_passes = 8 + 3;
    n_sorts = 2;
    extra = 3;
  } else if (sweep == 0) {
    const int nblk = (int)cdiv(nB, kCopyBlock);
    k_count_copies<<<nblk, kCopyBlock, 0, s>>>(nB, B, c->ctl);
    k_scan_copies<<<1, 1024, 0, s>>>(nblk, nB, B, c->ctl);
    k_expand_copies<<<grid, 256, 0, s>>>(nB, B, c->ctl, (unsigned long long *)B.keys[0], B.vals[0]);
    const int bits = sc.n > 0 ? 48 + sbits : 56;   // cell index: 16 bits batched, 24 bits alone
    // every pass of a digit the keys share is skipped; the gather finds the
    // result's buffers on the device and leaves the sorted keys in keys[0]
    const int *sel = nullptr;
    radix_sort(B.keys, B.vals, 8, B.cap_copies, c->sortw, s, &c->ctl->status, bits, &c->ctl->n_copies, &sel);
    const int cgrid = (int)std::min<int64_t>(cdiv(B.cap_copies, 256), (int64_t)c->sm_count * 8);
    k_gather_copies<<<cgrid, 256, 0, s>>>(nB, B, c->ctl, (unsigned long long *)B.keys[0],
                                          (const unsigned long long *)B.keys[1], B.vals[0], B.vals[1], sel);
    s_key = (const unsigned long long *)B.keys[0];
    sort_passes = (bits + 7) / 8;
    extra = 2;
  } else if (sc.n > 0) {
    // scene in the high word of the key: one sorted run per scene
    const int bits = 32 + sbits;
    k_make_keys_scenes<<<grid, 256, 0, s>>>(nB, B, (unsigned long long *)B.keys[0], B.vals[0]);
    const int cur = radix_sort(B.keys, B.vals, 8, nB, c->sortw, s, &c->ctl->status, bits);
    k_gather_sorted<<<grid, 256, 0, s>>>(nB, B.vals[cur], c->ctl, B);
    sort_passes = (bits + 7) / 8;
  } else if (!fp64) {
    k_make_keys<<<grid, 256, 0, s>>>(nB, B.lo32, c->ctl, (uint32_t *)B.keys[0], B.vals[0]);
    const int cur = radix_sort(B.keys, B.vals, 4, nB, c->sortw, s, &c->ctl->status);
    k_gather_sorted<<<grid, 256, 0, s>>>(nB, B.vals[cur], c->ctl, B);
  } else {
    k_make_keys64<<<grid, 256, 0, s>>>(nB, B.lo64, c->ctl, (unsigned long long *)B.keys[0], B.vals[0]);
    const int cur = radix_sort(B.keys, B.vals, 8, nB, c->sortw, s, &c->ctl->status);
    k_gather_sorted64<<<grid, 256, 0, s>>>(nB, B.vals[cur], c->ctl, B);
  }
  mark(c, CCD_STAGE_SORT, false, s);
  c->s_key_last = s_key;
  }

  SweepArgs A;
  A.nB = nB;
  A.nV = nV;
  A.nE = nE;
  A.n_scenes = sc.n;
  A.voff = sc.voff;
  A.eoff = sc.eoff;
  A.foff = sc.foff;
  A.bsid = c->bsid;
  A.s_alo = B.s_alo;
  A.s_ahi = B.s_ahi;
  A.s_oth = B.s_oth;
  A.s_vid = B.s_vid;
  A.s_tag = B.s_tag;
  A.s_alo64 = B.s_alo64;
  A.s_ahi64 = B.s_ahi64;
  A.s_oth64 = B.s_oth64;
  A.lo64 = B.lo64;
  A.hi64 = B.hi64;
  A.vf_out = vf_out;
  A.ee_out = ee_out;
  A.vf_cap = vf_cap;
  A.ee_cap = ee_cap;
  A.ee_rev = ee_rev ? 1 : 0;
  A.ctl = c->ctl;
  A.s_key = s_key;
  A.n_dev = &c->ctl->n_copies;
  A.sup = c->sup;
  A.sup_cap = c->sup_cap;
  A.i_begin = i_begin;
  A.i_end = i_end;
  const int sgrid = (int)std::min<int64_t>(cdiv(nB * 32, 256), (int64_t)c->sm_count * 32);
  if (phase & 2) {
  mark(c, CCD_STAGE_SWEEP, true, s);
  A.s_seg = B.s_seg;
  A.s_key64 = B.s_key64;
  A.s_ahi64c = B.s_ahi64c;
  A.s_oth64c = B.s_oth64c;
  if (strips64) {
    k_sweep_strips64<<<(unsigned)std::min<int64_t>(cdiv(B.cap_copies, 256), (int64_t)c->sm_count * 16), 128, 0, s>>>(
        A);
    k_exact_filter<<<(unsigned)std::min<int64_t>(cdiv(c->sup_cap, 2048), (int64_t)c->sm_count * 8), 256, 0, s>>>(A);
    extra += 1;
  } else if (fp64)
    k_sweep64<<<sgrid, 256, 0, s>>>(A);
  else if (sweep == 1)
    k_sweep<<<sgrid, 256, 0, s>>>(A);
  else if (sweep == 2)
    k_sweep_tiled<<<(unsigned)cdiv(nB, 256), 128, 0, s>>>(A);
  else {
    k_sweep_strips<<<(unsigned)std::min<int64_t>(cdiv(B.cap_copies, 256), (int64_t)c->sm_count * 16), 128, 0, s>>>(A);
    k_exact_filter<<<(unsigned)std::min<int64_t>(cdiv(c->sup_cap, 2048), (int64_t)c->sm_count * 8), 256, 0, s>>>(A);
    extra += 1;
  }
  mark(c, CCD_STAGE_SWEEP, false, s);
  }
  // reset, build, axis, keys (or count, scan, expand), per sort a counting
  // kernel and one kernel per pass (skipped passes included: they return at
  // once), gather, sweep (and exact filter)
  c->n_launches += (phase & 1 ? 5 : 1) + (phase & 2 ? 1 : 0) + extra + n_sorts + sort_passes;
  CK(cudaGetLastError());
  return CCD_OK;
}

// The per-primitive set-up alone (needs only the mesh), e.g. on a side stream
// beside the broad phase.
int launch_prims(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                 const int32_t *F, int64_t nF, cudaStream_t s) {
  const int64_t nP = nV + nE + nF;
  if (nP == 0) return CCD_OK;
  if (narrow_prim_words(nV, nE, nF) > c->cap_prims) return CCD_EINVAL;   // sized before
  NarrowArgs A;
  std::memset(&A, 0, sizeof(A));
  A.ctl = c->ctl;
  A.V0 = V0;
  A.V1 = V1;
  A.nV = nV;
  A.nE = nE;
  A.nF = nF;
  A.E = E;
  A.F = F;
  A.prims = c->prims;
  k_prepare_prims<<<(unsigned)std::min<int64_t>(cdiv(nP, 256), (int64_t)c->sm_count * 16), 256, 0, s>>>(A);
  c->n_launches += 1;
  CK(cudaGetLastError());
  return CCD_OK;
}

int launch_narrow(ccd_ctx *c, const int32_t *vf, int64_t n_vf, const int32_t *ee, int64_t n_ee,
                  int counts_from_ctl, const double *V0, const double *V1, int64_t nV, const int32_t *E,
                  int64_t nE, const int32_t *F, int64_t nF, double delta, double min_sep, int64_t max_iter, int mode,
                  unsigned long long *toi_vf_bits, unsigned long long *toi_ee_bits, cudaStream_t s,
                  bool zero_rule_pass = false, int n_scenes = 0, const int64_t *voff = nullptr,
                  unsigned long long *toi_scene = nullptr, int64_t ee_end = 0, bool keep_toi = false,
                  unsigned long long phantom_units = 0, bool prims_done = false) {
  const int64_t nq = counts_from_ctl && ee_end > 0 ? ee_end : n_vf + n_ee;
  int rc = ensure_narrow(c, nq, s);
  if (rc) return rc;
  const int64_t nP = nV + nE + nF;
  if (narrow_prim_words(nV, nE, nF) > c->cap_prims) {
    if (c->capturing) return CCD_EINVAL;   // (buffers are sized before a capture)
    rc = ensure_prims(c, nV, nE, nF);
    if (rc) return rc;
  }
  if (zero_rule_pass)
    k_nozero_prepare<<<1, 1, 0, s>>>(c->ctl);
  else
    k_reset_narrow<<<1, 1, 0, s>>>(c->ctl, keep_toi ? 1 : 0);
  if (phantom_units) k_add_pending<<<1, 1, 0, s>>>(c->ctl, phantom_units);   // self-test only
  NarrowArgs A;
  A.ctl = c->ctl;
  A.vf = vf;
  A.ee = ee;
  A.n_vf = n_vf;
  A.n_ee = n_ee;
  A.counts_from_ctl = counts_from_ctl;
  A.ee_end = ee_end;
  A.V0 = V0;
  A.V1 = V1;
  A.nV = nV;
  A.nE = nE;
  A.nF = nF;
  A.E = E;
  A.F = F;
  A.prims = c->prims;
  A.delta = delta;
  A.min_sep = min_sep;
  A.max_iter = max_iter;
  A.mode = mode;
  A.budget = c->opts.export_budget > 0 ? c->opts.export_budget : 16;
  A.no_zero = zero_rule_pass ? 1 : 0;
  A.only_if_rerun = zero_rule_pass ? 1 : 0;
  A.toi_vf_bits = toi_vf_bits;
  A.toi_ee_bits = toi_ee_bits;
  A.qflags = c->qflags;
  A.qiters = c->qiters;
  A.ring = c->ring;
  A.ring_mask = c->ring_cap - 1;
  A.qrec = c->qrec;
  A.rec_stride = c->cap_q;
  A.n_scenes = n_scenes;
  A.voff = voff;
  A.toi_scene = toi_scene;
  A.qsid = c->qsid;
  if (!zero_rule_pass) mark(c, CCD_STAGE_NARROW, true, s);
  // per-primitive set-up (independent of min_sep: the zero-TOI pass reuses
  // it), then the query records in one dense pass (the zero-TOI pass has
  // min_sep = 0: redo them)
  const bool prims = !zero_rule_pass && !prims_done && nP > 0;
  if (prims)
    k_prepare_prims<<<(unsigned)std::min<int64_t>(cdiv(nP, 256), (int64_t)c->sm_count * 16), 256, 0, s>>>(A);
  k_prepare_queries<<<(unsigned)std::min<int64_t>(cdiv(std::max<int64_t>(nq, 1), 256), (int64_t)c->sm_count * 16),
                      256, 0, s>>>(A);
  if (!zero_rule_pass) mark(c, CCD_STAGE_NARROW_KERNEL, true, s);
  k_narrow<<<c->narrow_blocks, kNarrowThreads, kNarrowDynSmem, s>>>(A);
  if (!zero_rule_pass) mark(c, CCD_STAGE_NARROW_KERNEL, false, s);
  if (zero_rule_pass) k_nozero_finish<<<1, 1, 0, s>>>(c->ctl);
  mark(c, CCD_STAGE_NARROW, false, s);
  // reset/prepare, primitives, records, narrow, finish
  c->n_launches += (zero_rule_pass ? 4 : 3) + (prims ? 1 : 0);
  CK(cudaGetLastError());
  return CCD_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Replay the graph cached for `key`, or capture `enqueue` on the private
// stream into a new one.  Buffers must already have their sizes: nothing may
// allocate while a capture is open.
template <class Enqueue>
int run_graph(ccd_ctx *c, ccd_ctx::GraphEntry &g, const void *key, size_t key_len, cudaStream_t s,
              Enqueue enqueue) {
  if (g.valid && std::memcmp(g.key, key, key_len) == 0) {
    CK(cudaGraphLaunch(g.exec, s));
    c->n_launches += g.launches;
    return CCD_OK;
  }
  if (g.valid) {
    cudaGraphExecDestroy(g.exec);
    g.valid = false;
  }
  if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  const long long before = c->n_launches;
  CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeRelaxed));
  c->capturing = true;
  const int rc = enqueue(c->cap_stream);
  c->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->cap_stream, &graph);
  if (rc != CCD_OK || e != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return rc != CCD_OK ? rc : CCD_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return CCD_ECUDA;
  std::memcpy(g.key, key, key_len);
  g.valid = true;
  g.launches = c->n_launches - before;
  CK(cudaGraphLaunch(g.exec, s));
  return CCD_OK;
}

}  // namespace

extern "C" {

void ccd_default_opts(ccd_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->delta = 1e-6;
  o->min_sep = 0.0;
  o->max_iter = 1000000;
  o->broad_fp64 = 0;
  o->sweep_kernel = 0;
  o->pair_capacity = 0;
  o->queue_capacity = 0;
  o->export_budget = 0;
  o->profile_stages = 0;
  o->no_zero_toi = 0;
  o->use_graph = 0;
}

int ccd_create(ccd_ctx **out, const ccd_opts *o, int device) {
  if (!out) return CCD_EINVAL;
  *out = nullptr;
  ccd_opts opts;
  ccd_default_opts(&opts);
  if (o) opts = *o;
  if (!(opts.delta >= 0) || !(opts.min_sep >= 0) || opts.max_iter < 0) return CCD_EINVAL;
  if (opts.broad_fp64 != 0 && opts.broad_fp64 != 1) return CCD_EINVAL;
  if (opts.sweep_kernel < 0 || opts.sweep_kernel > 2 || !(opts.strip_width >= 0)) return CCD_EINVAL;
  if (opts.no_zero_toi != 0 && opts.no_zero_toi != 1) return CCD_EINVAL;
  if (opts.use_graph != 0 && opts.use_graph != 1) return CCD_EINVAL;
  if (opts.profile_stages != 0 && opts.profile_stages != 1) return CCD_EINVAL;
  if (opts.queue_capacity < 0 || (opts.queue_capacity & (opts.queue_capacity - 1))) return CCD_EINVAL;
  int ndev = 0;
  CK(cudaGetDeviceCount(&ndev));
  if (device < 0 || device >= ndev) return CCD_EINVAL;
  cudaDeviceProp p;
  CK(cudaGetDeviceProperties(&p, device));
  if (p.major != 10 || p.minor != 3) return CCD_EDEVICE;
  CK(cudaSetDevice(device));
  ccd_ctx *c = new (std::nothrow) ccd_ctx();
  if (!c) return CCD_ENOMEM;
  c->device = device;
  c->opts = opts;
  c->sm_count = p.multiProcessorCount;
  int per_sm = 0;
  if (cudaFuncSetAttribute(k_narrow, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kNarrowDynSmem) !=
      cudaSuccess) {
    delete c;
    return CCD_ECUDA;
  }
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow, kNarrowThreads, kNarrowDynSmem) !=
          cudaSuccess ||
      per_sm < 1)
    per_sm = 1;
  c->narrow_blocks = per_sm * c->sm_count;
  if (cudaMalloc(&c->ctl, sizeof(DevCtl)) != cudaSuccess) {
    delete c;
    return CCD_ENOMEM;
  }
  cudaMemset(c->ctl, 0, sizeof(DevCtl));
  if (opts.profile_stages)
    for (int k = 0; k < 2 * CCD_NSTAGES; ++k)
      if (cudaEventCreate(&c->ev[k]) != cudaSuccess) {
        cudaFree(c->ctl);
        delete c;
        return CCD_ECUDA;
      }
  *out = c;
  return CCD_OK;
}

int ccd_destroy(ccd_ctx *c) {
  if (!c) return CCD_EINVAL;
  cudaSetDevice(c->device);
  cudaDeviceSynchronize();
  cudaFree(c->broad_mem);
  cudaFree(c->vf);
  cudaFree(c->sup);
  cudaFree(c->qflags);
  cudaFree(c->qiters);
  cudaFree(c->qrec);
  cudaFree(c->qsid);
  cudaFree(c->prims);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  cudaFree(c->bsid);
  cudaFree(c->ssum);
  cudaFree(c->saxis);
  cudaFree(c->smm);
  cudaFree(c->strips64_mem);
  cudaFree(c->sparam_sc);
  cudaFree(c->ring);
  if (c->g_step.valid) cudaGraphExecDestroy(c->g_step.exec);
  if (c->g_batch.valid) cudaGraphExecDestroy(c->g_batch.exec);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  cudaFree(c->ctl);
  for (int k = 0; k < 2 * CCD_NSTAGES; ++k)
    if (c->ev[k]) cudaEventDestroy(c->ev[k]);
  delete c;
  return CCD_OK;
}

int ccd_broad(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
              const int32_t *F, int64_t nF, int32_t *vf_out, int64_t vf_cap, int64_t *n_vf, int32_t *ee_out,
              int64_t ee_cap, int64_t *n_ee, void *stream) {
  if (!c || !n_vf || !n_ee || vf_cap < 0 || ee_cap < 0) return CCD_EINVAL;
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  if ((vf_cap > 0 && !vf_out) || (ee_cap > 0 && !ee_out)) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  clear_marks(c);
  k_reset_status<<<1, 1, 0, s>>>(c->ctl);
  c->n_launches += 1;
  int rc = launch_broad(c, V0, V1, nV, E, nE, F, nF, vf_out, vf_cap, ee_out, ee_cap, s);
  if (rc) return rc;
  unsigned long long h[3];
  int ovf = 0;
  CK(cudaMemcpyAsync(h, &c->ctl->n_vf, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&ovf, &c->ctl->sup_overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n_vf = (int64_t)h[0];
  *n_ee = (int64_t)h[1];
  if (ovf) {
    // the candidates did not all fit: their count bounds both lists
    *n_vf = std::max<int64_t>(*n_vf, (int64_t)h[2]);
    *n_ee = std::max<int64_t>(*n_ee, (int64_t)h[2]);
    return CCD_ETRUNC;
  }
  return ((int64_t)h[0] > vf_cap || (int64_t)h[1] > ee_cap) ? CCD_ETRUNC : CCD_OK;
}

int ccd_broad_shard(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                    const int32_t *F, int64_t nF, int32_t shard, int32_t n_shards, int32_t *vf_out, int64_t vf_cap,
                    int64_t *n_vf, int32_t *ee_out, int64_t ee_cap, int64_t *n_ee, void *stream) {
  if (!c || !n_vf || !n_ee || vf_cap < 0 || ee_cap < 0 || n_shards < 1 || shard < 0 || shard >= n_shards)
    return CCD_EINVAL;
  if (c->opts.sweep_kernel != 0) return CCD_EINVAL;   // sweep ranges exist in the cell sweep only
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  if ((vf_cap > 0 && !vf_out) || (ee_cap > 0 && !ee_out)) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  clear_marks(c);
  k_reset_status<<<1, 1, 0, s>>>(c->ctl);
  c->n_launches += 1;
  // boxes, cell copies and sort (every shard does the same, small work) ...
  int rc = launch_broad(c, V0, V1, nV, E, nE, F, nF, vf_out, vf_cap, ee_out, ee_cap, s,
                        SceneSpec{0, nullptr, nullptr, nullptr}, false, 1);
  if (rc) return rc;
  unsigned long long ncopy = 0;
  CK(cudaMemcpyAsync(&ncopy, &c->ctl->n_copies, sizeof(ncopy), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  // ... then the sweep from this shard's contiguous part of the sorted
  // copies (it reads past the part's end; every pair is reported from one
  // copy, so the shards' pair sets are disjoint and cover the whole set)
  const int64_t b = (int64_t)(ncopy * (unsigned long long)shard / (unsigned long long)n_shards);
  const int64_t e = (int64_t)(ncopy * (unsigned long long)(shard + 1) / (unsigned long long)n_shards);
  rc = launch_broad(c, V0, V1, nV, E, nE, F, nF, vf_out, vf_cap, ee_out, ee_cap, s,
                    SceneSpec{0, nullptr, nullptr, nullptr}, false, 2, b, e);
  if (rc) return rc;
  unsigned long long h[3];
  int ovf = 0;
  CK(cudaMemcpyAsync(h, &c->ctl->n_vf, sizeof(h), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&ovf, &c->ctl->sup_overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *n_vf = (int64_t)h[0];
  *n_ee = (int64_t)h[1];
  if (ovf) {
    *n_vf = std::max<int64_t>(*n_vf, (int64_t)h[2]);
    *n_ee = std::max<int64_t>(*n_ee, (int64_t)h[2]);
    return CCD_ETRUNC;
  }
  return ((int64_t)h[0] > vf_cap || (int64_t)h[1] > ee_cap) ? CCD_ETRUNC : CCD_OK;
}

int ccd_narrow(ccd_ctx *c, const int32_t *vf, int64_t n_vf, const int32_t *ee, int64_t n_ee, const double *V0,
               const double *V1, int64_t nV, const int32_t *E, int64_t nE, const int32_t *F, int64_t nF,
               double delta, double min_sep, int64_t max_iter, int32_t mode, double *toi_vf, double *toi_ee,
               uint8_t *flags_vf, uint8_t *flags_ee, double *toi_min, void *stream) {
  if (!c || n_vf < 0 || n_ee < 0 || !toi_min || (mode != 0 && mode != 1)) return CCD_EINVAL;
  if (!(delta >= 0) || !(min_sep >= 0) || max_iter < 0) return CCD_EINVAL;
  if ((n_vf > 0 && (!vf || !F)) || (n_ee > 0 && (!ee || !E))) return CCD_EINVAL;
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  if (mode == 0 && ((n_vf > 0 && !toi_vf) || (n_ee > 0 && !toi_ee))) return CCD_EINVAL;
  if (n_vf + n_ee >= (1ll << 32)) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  clear_marks(c);
  k_reset_status<<<1, 1, 0, s>>>(c->ctl);
  c->n_launches += 1;
  int rc = ensure_narrow(c, n_vf + n_ee, s);
  if (rc) return rc;
  // mode 1 keeps no per-pair results
  unsigned long long *tv = mode == 0 ? (unsigned long long *)toi_vf : nullptr;
  unsigned long long *te = mode == 0 ? (unsigned long long *)toi_ee : nullptr;
  const int g = (int)std::min<int64_t>(cdiv(std::max<int64_t>(n_vf + n_ee, 1), 256), (int64_t)c->sm_count * 8);
  rc = launch_narrow(c, vf, n_vf, ee, n_ee, 0, V0, V1, nV, E, nE, F, nF, delta, min_sep, max_iter, mode, tv, te, s);
  if (rc) return rc;
  if (mode == 0 && n_vf + n_ee > 0) {
    k_flags_out<<<g, 256, 0, s>>>(c->qflags, n_vf, n_ee, flags_vf, flags_ee, c->ctl);
    c->n_launches += 1;
  }
  CK(cudaMemcpyAsync(toi_min, &c->ctl->toi_bits, sizeof(double), cudaMemcpyDeviceToDevice, s));
  CK(cudaGetLastError());
  return CCD_OK;
}

}  // extern "C"

namespace {

// The paper's batching for one scene whose candidate pairs do not fit the
// memory limit: boxes and sort once, then the sweep over ranges of the
// sorted copies, each range's pairs narrowed with the earliest time carried
// over; a range whose pairs overflow is halved.  Synchronous.
int ranged_step(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                const int32_t *F, int64_t nF, double delta, double min_sep, int64_t max_iter, unsigned long long need,
                double *toi_min, cudaStream_t s) {
  if (c->opts.sweep_kernel != 0 || c->opts.no_zero_toi) return CCD_ETRUNC;
  const int64_t cap = c->pair_cap;
  clear_marks(c);
  k_reset_status<<<1, 1, 0, s>>>(c->ctl);
  int rc = launch_broad(c, V0, V1, nV, E, nE, F, nF, c->vf, cap, c->ee, cap, s,
                        SceneSpec{0, nullptr, nullptr, nullptr}, true, 1);
  if (rc) return rc;
  unsigned long long ncopy = 0;
  CK(cudaMemcpyAsync(&ncopy, &c->ctl->n_copies, sizeof(ncopy), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  const int64_t k0 = std::max<int64_t>(2, (int64_t)(need / (unsigned long long)std::max<int64_t>(1, cap * 3 / 4)) + 1);
  std::vector<std::pair<int64_t, int64_t>> todo;
  for (int64_t k = k0 - 1; k >= 0; --k)
    todo.push_back({(int64_t)ncopy * k / k0, (int64_t)ncopy * (k + 1) / k0});
  bool first = true;
  int64_t ranges = 0;
  while (!todo.empty()) {
    const auto r = todo.back();
    todo.pop_back();
    if (r.first >= r.second) continue;
    rc = launch_broad(c, V0, V1, nV, E, nE, F, nF, c->vf, cap, c->ee, cap, s, SceneSpec{0, nullptr, nullptr, nullptr},
                      true, 2, r.first, r.second);
    if (rc) return rc;
    struct {
      unsigned long long nvf, nee, nsup;
      int ovf;
    } h;
    CK(cudaMemcpyAsync(&h.nvf, &c->ctl->n_vf, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h.ovf, &c->ctl->sup_overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (h.ovf || (int64_t)(h.nvf + h.nee) > cap) {
      if (r.second - r.first <= 1) return CCD_ETRUNC;   // one box's pairs alone do not fit
      const int64_t m = (r.first + r.second) / 2;
      todo.push_back({m, r.second});
      todo.push_back({r.first, m});
      continue;
    }
    k_counts_from_broad<<<1, 1, 0, s>>>(c->ctl, cap);
    c->n_launches += 1;
    rc = launch_narrow(c, c->vf, cap, c->ee, cap, 1, V0, V1, nV, E, nE, F, nF, delta, min_sep, max_iter, 1, nullptr,
                       nullptr, s, false, 0, nullptr, nullptr, cap, !first);
    if (rc) return rc;
    first = false;
    ++ranges;
  }
  c->last_ranges = ranges;
  struct {
    unsigned long long toi;
    int status;
  } h;
  CK(cudaMemcpyAsync(&h.toi, &c->ctl->toi_bits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(&h.status, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  std::memcpy(toi_min, &h.toi, sizeof(double));
  return h.status;
}

}  // namespace

extern "C" {

int ccd_step(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
             const int32_t *F, int64_t nF, double delta, double min_sep, int64_t max_iter, double *toi_min,
             void *stream) {
  if (!c || !toi_min || !(delta >= 0) || !(min_sep >= 0) || max_iter < 0) return CCD_EINVAL;
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  const bool host_out = !is_device_ptr(toi_min);
  int64_t want = c->opts.pair_capacity > 0 ? c->opts.pair_capacity : default_pair_capacity(nV + nE + nF);
  int64_t limit_cap = INT64_MAX;   // pair capacity that fits opts.memory_limit
  if (c->opts.memory_limit > 0) {
    limit_cap = ccd_pair_capacity_for(&c->opts, c->opts.memory_limit, nV + nE + nF, 0);
    if (limit_cap < 1024) return CCD_ENOMEM;
    want = std::min(want, limit_cap);
  }
  c->last_ranges = 0;
  auto enqueue = [&](cudaStream_t st) -> int {
    clear_marks(c);
    k_reset_status<<<1, 1, 0, st>>>(c->ctl);
    // the per-primitive set-up of the narrow phase needs only the mesh: it
    // runs on a side stream beside the broad phase and joins before the
    // query records are built
    CK(cudaEventRecord(c->ev_fork, st));
    CK(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
    int r = launch_prims(c, V0, V1, nV, E, nE, F, nF, c->side);
    if (r) return r;
    CK(cudaEventRecord(c->ev_join, c->side));
    r = launch_broad(c, V0, V1, nV, E, nE, F, nF, c->vf, c->pair_cap, c->ee, c->pair_cap, st,
                     SceneSpec{0, nullptr, nullptr, nullptr}, true);
    if (r) return r;
    k_counts_from_broad<<<1, 1, 0, st>>>(c->ctl, c->pair_cap);
    c->n_launches += 2;
    CK(cudaStreamWaitEvent(st, c->ev_join, 0));
    r = launch_narrow(c, c->vf, c->pair_cap, c->ee, c->pair_cap, 1, V0, V1, nV, E, nE, F, nF, delta, min_sep, max_iter, 1,
                      nullptr, nullptr, st, false, 0, nullptr, nullptr, c->pair_cap, false, 0, true);
    if (r) return r;
    if (c->opts.no_zero_toi) {
      // second pass only when the first found t* = 0 (decided on the device)
      r = launch_narrow(c, c->vf, c->pair_cap, c->ee, c->pair_cap, 1, V0, V1, nV, E, nE, F, nF, delta, 0.0, max_iter, 1,
                        nullptr, nullptr, st, true, 0, nullptr, nullptr, c->pair_cap);
      if (r) return r;
    }
    if (!host_out && cudaMemcpyAsync(toi_min, &c->ctl->toi_bits, sizeof(double), cudaMemcpyDeviceToDevice, st) !=
                         cudaSuccess)
      return CCD_ECUDA;
    return CCD_OK;
  };
  for (int attempt = 0; attempt < 3; ++attempt) {
    int rc = ensure_pairs(c, want);
    if (rc) return rc;
    rc = ensure_narrow(c, c->pair_cap, s);
    if (rc) return rc;
    rc = ensure_prims(c, nV, nE, nF);
    if (rc) return rc;
    if (!c->side) {
      CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
      CK(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    }
    rc = ensure_broad(c, nV + nE + nF);
    if (rc) return rc;
    if (c->opts.broad_fp64 && c->opts.sweep_kernel == 0) {
      rc = ensure_strips64(c);
      if (rc) return rc;
    }
    if (!host_out) {
      if (!c->opts.use_graph) return enqueue(s);
      struct {
        const void *p[6];
        int64_t n[4];
        double d[2];
        int64_t mi;
      } key;
      std::memset(&key, 0, sizeof(key));
      key.p[0] = V0; key.p[1] = V1; key.p[2] = E; key.p[3] = F; key.p[4] = toi_min; key.p[5] = c->vf;
      key.n[0] = nV; key.n[1] = nE; key.n[2] = nF; key.n[3] = c->pair_cap;
      key.d[0] = delta; key.d[1] = min_sep;
      key.mi = max_iter;
      return run_graph(c, c->g_step, &key, sizeof(key), s, enqueue);
    }
    rc = enqueue(s);
    if (rc) return rc;
    struct {
      unsigned long long nvf, nee, nsup, toi;
      int status, ovf;
    } h;
    CK(cudaMemcpyAsync(&h.nvf, &c->ctl->n_vf, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h.toi, &c->ctl->toi_bits, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h.status, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&h.ovf, &c->ctl->sup_overflow, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (!h.ovf && (int64_t)(h.nvf + h.nee) <= c->pair_cap) {
      std::memcpy(toi_min, &h.toi, sizeof(double));
      return h.status;
    }
    // the candidate buffer holds twice the pair capacity
    unsigned long long need = h.nvf + h.nee;
    if (h.ovf) need = std::max(need, h.nsup / 2 + 1);
    if ((int64_t)need > limit_cap - limit_cap / 8 - 1024 || c->pair_cap >= limit_cap)
      return ranged_step(c, V0, V1, nV, E, nE, F, nF, delta, min_sep, max_iter, need, toi_min, s);
    want = std::min<int64_t>((int64_t)need + (int64_t)(need / 8) + 1024, limit_cap);
  }
  return CCD_ETRUNC;
}

int ccd_step_batch(ccd_ctx *c, int32_t n_scenes, const int64_t *vert_off, const int64_t *edge_off,
                   const int64_t *face_off, const double *V0, const double *V1, int64_t nV, const int32_t *E,
                   int64_t nE, const int32_t *F, int64_t nF, double delta, double min_sep, int64_t max_iter,
                   double *toi_out, void *stream) {
  if (!c || n_scenes < 1 || !vert_off || !edge_off || !face_off || !toi_out) return CCD_EINVAL;
  if (!(delta >= 0) || !(min_sep >= 0) || max_iter < 0) return CCD_EINVAL;
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  if (c->opts.broad_fp64 != 0 || c->opts.sweep_kernel == 1 || c->opts.no_zero_toi != 0) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  clear_marks(c);
  const int64_t nB = nV + nE + nF;
  int rc = ensure_pairs(c, c->opts.pair_capacity > 0 ? c->opts.pair_capacity : default_pair_capacity(nB));
  if (rc) return rc;
  rc = ensure_narrow(c, c->pair_cap, s);
  if (rc) return rc;
  rc = ensure_prims(c, nV, nE, nF);
  if (rc) return rc;
  rc = ensure_broad(c, nB);
  if (rc) return rc;
  rc = ensure_scenes(c, nB, n_scenes);
  if (rc) return rc;
  auto enqueue = [&](cudaStream_t st) -> int {
    clear_marks(c);
    k_reset_status<<<1, 1, 0, st>>>(c->ctl);
    const SceneSpec sc{n_scenes, vert_off, edge_off, face_off};
    int r = launch_broad(c, V0, V1, nV, E, nE, F, nF, c->vf, c->pair_cap, c->ee, c->pair_cap, st, sc, true);
    if (r) return r;
    k_counts_from_broad<<<1, 1, 0, st>>>(c->ctl, c->pair_cap);
    k_fill_u64<<<(unsigned)std::min<int64_t>(cdiv(n_scenes, 256), 1024), 256, 0, st>>>(
        (unsigned long long *)toi_out, n_scenes, 0x7FF0000000000000ull);
    c->n_launches += 3;
    return launch_narrow(c, c->vf, c->pair_cap, c->ee, c->pair_cap, 1, V0, V1, nV, E, nE, F, nF, delta, min_sep, max_iter,
                         2, nullptr, nullptr, st, false, n_scenes, vert_off, (unsigned long long *)toi_out,
                         c->pair_cap);
  };
  if (!c->opts.use_graph) return enqueue(s);
  struct {
    const void *p[9];
    int64_t n[5];
    double d[2];
    int64_t mi;
  } key;
  std::memset(&key, 0, sizeof(key));
  key.p[0] = V0; key.p[1] = V1; key.p[2] = E; key.p[3] = F; key.p[4] = toi_out;
  key.p[5] = vert_off; key.p[6] = edge_off; key.p[7] = face_off; key.p[8] = c->vf;
  key.n[0] = nV; key.n[1] = nE; key.n[2] = nF; key.n[3] = n_scenes; key.n[4] = c->pair_cap;
  key.d[0] = delta; key.d[1] = min_sep;
  key.mi = max_iter;
  return run_graph(c, c->g_batch, &key, sizeof(key), s, enqueue);
}

}  // extern "C"

namespace {

// The autotuner on one scene (sc.n == 0) or on batched scenes.
int autotune_impl(ccd_ctx *c, const SceneSpec &sc, const double *V0, const double *V1, int64_t nV,
                  const int32_t *E, int64_t nE, const int32_t *F, int64_t nF, int32_t reps, ccd_tuning *out,
                  void *stream) {
  if (!c || !out || reps < 1 || c->opts.broad_fp64 != 0) return CCD_EINVAL;
  if (!mesh_args_ok(V0, V1, nV, E, nE, F, nF)) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const ccd_opts saved = c->opts;
  const bool graph = c->opts.use_graph != 0;
  c->opts.use_graph = 0;
  std::memset(out, 0, sizeof(*out));
  // one step sizes every buffer (pairs grow to fit)
  unsigned long long *toi_sc = nullptr;   // per-scene earliest times (batched scenes)
  int rc = CCD_OK;
  if (sc.n > 0) {
    CK(cudaMalloc(&toi_sc, sc.n * sizeof(double)));
    rc = ccd_step_batch(c, sc.n, sc.voff, sc.eoff, sc.foff, V0, V1, nV, E, nE, F, nF, c->opts.delta,
                        c->opts.min_sep, c->opts.max_iter, (double *)toi_sc, stream);
    if (rc == CCD_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = CCD_ECUDA;
  } else {
    double t0 = 0.0;
    rc = ccd_step(c, V0, V1, nV, E, nE, F, nF, c->opts.delta, c->opts.min_sep, c->opts.max_iter, &t0, stream);
  }
  if (rc) {
    c->opts = saved;
    cudaFree(toi_sc);
    return rc;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int err = CCD_OK;
  int trials = 0;
  // median of `reps` timings of one phase; the broad phase leaves its pairs
  // in the context's buffers for the narrow phase
  auto timed = [&](bool narrow) -> double {
    double v[16];
    const int n = std::min(reps, 16);
    for (int r = 0; r < n; ++r) {
      if (narrow) {
        k_reset_status<<<1, 1, 0, s>>>(c->ctl);
        k_counts_from_broad<<<1, 1, 0, s>>>(c->ctl, c->pair_cap);
      }
      cudaEventRecord(e0, s);
      if (narrow && sc.n > 0)
        k_fill_u64<<<(unsigned)std::min<int64_t>(cdiv(sc.n, 256), 1024), 256, 0, s>>>(toi_sc, sc.n,
                                                                                     0x7FF0000000000000ull);
      int r2 = narrow ? launch_narrow(c, c->vf, c->pair_cap, c->ee, c->pair_cap, 1, V0, V1, nV, E, nE, F, nF,
                                      c->opts.delta, c->opts.min_sep, c->opts.max_iter, sc.n > 0 ? 2 : 1, nullptr,
                                      nullptr, s, false, sc.n, sc.voff, toi_sc, c->pair_cap)
                      : launch_broad(c, V0, V1, nV, E, nE, F, nF, c->vf, c->pair_cap, c->ee, c->pair_cap, s, sc,
                                     true);
      cudaEventRecord(e1, s);
      if (cudaStreamSynchronize(s) != cudaSuccess) r2 = CCD_ECUDA;
      int st = CCD_OK;
      if (cudaMemcpy(&st, &c->ctl->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) r2 = CCD_ECUDA;
      if (r2 || st) {
        err = r2 ? r2 : st;
        return 1e30;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      v[r] = ms;
    }
    ++trials;
    std::sort(v, v + n);
    return v[n / 2];
  };
  // 1. sweep: strips of several widths, or one sorted list
  const double widths[] = {1.5, 2.0, 3.0, 4.0, 6.0};
  double best_b = 1e30;
  int best_sweep = 0;
  double best_w = 2.0;
  c->opts.sweep_kernel = saved.sweep_kernel;
  c->opts.strip_width = saved.strip_width;
  const double base_b = timed(false);
  for (double w : widths) {
    c->opts.sweep_kernel = 0;
    c->opts.strip_width = w;
    const double t = timed(false);
    if (t < best_b) { best_b = t; best_sweep = 0; best_w = w; }
  }
  c->opts.sweep_kernel = 2;
  {
    const double t = timed(false);
    if (t < best_b) { best_b = t; best_sweep = 2; best_w = 0.0; }
  }
  c->opts.sweep_kernel = best_sweep;
  c->opts.strip_width = best_w;
  timed(false);   // pairs of the chosen sweep for the narrow trials
  // 2. narrow: intervals between hand-offs in the tail phase
  const int budgets[] = {8, 16, 32, 64};
  c->opts.export_budget = saved.export_budget;
  const double base_n = timed(true);
  double best_n = 1e30;
  int best_budget = 16;
  long long peak = 0;
  for (int b : budgets) {
    c->opts.export_budget = b;
    const double t = timed(true);
    unsigned long long qp = 0;
    cudaMemcpy(&qp, &c->ctl->queue_peak, sizeof(qp), cudaMemcpyDeviceToHost);
    peak = std::max<long long>(peak, (long long)qp);
    if (t < best_n) { best_n = t; best_budget = b; }
  }
  c->opts.export_budget = best_budget;
  // 3. queue: the smallest power of two with 16x headroom over the peak
  // occupancy seen (hand-offs stop at a quarter of the capacity), kept if the
  // narrow phase is not slower by more than 2%
  unsigned long long qcap = 1024;
  while (qcap < 16ull * (unsigned long long)peak) qcap <<= 1;
  if (err == CCD_OK && qcap < c->ring_cap) {
    const unsigned long long old_cap = c->ring_cap;
    auto regrow = [&](unsigned long long cap) -> int {
      CK(cudaStreamSynchronize(s));
      CK(cudaFree(c->ring));
      c->ring = nullptr;
      c->ring_cap = 0;
      c->opts.queue_capacity = (int64_t)cap;
      return ensure_narrow(c, 0, s);
    };
    rc = regrow(qcap);
    if (rc) err = rc;
    const double t = err ? 1e30 : timed(true);
    if (t <= 1.02 * best_n) {
      best_n = std::min(best_n, t);
    } else if (err == CCD_OK) {
      rc = regrow(old_cap);
      if (rc) err = rc;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (toi_sc) {
    cudaStreamSynchronize(s);
    cudaFree(toi_sc);
    toi_sc = nullptr;
  }
  // launch configurations changed: captured graphs are stale
  if (c->g_step.valid) { cudaGraphExecDestroy(c->g_step.exec); c->g_step.valid = false; }
  if (c->g_batch.valid) { cudaGraphExecDestroy(c->g_batch.exec); c->g_batch.valid = false; }
  c->opts.use_graph = graph ? 1 : 0;
  if (err) {
    const ccd_opts keep = c->opts;
    c->opts = saved;
    c->opts.queue_capacity = keep.queue_capacity;   // the ring as it stands
    return err;
  }
  c->opts.queue_capacity = (int64_t)c->ring_cap;
  out->sweep_kernel = c->opts.sweep_kernel;
  out->export_budget = c->opts.export_budget;
  out->strip_width = c->opts.strip_width;
  out->queue_capacity = (int64_t)c->ring_cap;
  out->broad_ms = best_b;
  out->narrow_ms = best_n;
  out->default_ms = base_b + base_n;
  out->n_trials = trials;
  return CCD_OK;
}

}  // namespace

extern "C" {

int ccd_autotune(ccd_ctx *c, const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                 const int32_t *F, int64_t nF, int32_t reps, ccd_tuning *out, void *stream) {
  return autotune_impl(c, SceneSpec{0, nullptr, nullptr, nullptr}, V0, V1, nV, E, nE, F, nF, reps, out, stream);
}

int ccd_autotune_batch(ccd_ctx *c, int32_t n_scenes, const int64_t *vert_off, const int64_t *edge_off,
                       const int64_t *face_off, const double *V0, const double *V1, int64_t nV, const int32_t *E,
                       int64_t nE, const int32_t *F, int64_t nF, int32_t reps, ccd_tuning *out, void *stream) {
  if (n_scenes < 1 || !vert_off || !edge_off || !face_off) return CCD_EINVAL;
  return autotune_impl(c, SceneSpec{n_scenes, vert_off, edge_off, face_off}, V0, V1, nV, E, nE, F, nF, reps, out,
                       stream);
}

int ccd_status_async(ccd_ctx *c, int32_t *status, void *stream) {
  if (!c || !status) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(cudaMemcpyAsync(status, &c->ctl->status, sizeof(int32_t), cudaMemcpyDefault, (cudaStream_t)stream));
  return CCD_OK;
}

int ccd_selftest_unfinished_work(ccd_ctx *c, int32_t *status, void *stream) {
  if (!c || !status) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  c->last_stream = s;
  k_reset_status<<<1, 1, 0, s>>>(c->ctl);
  // no queries, and one unit counted as pending that no lane will ever take
  const int rc = launch_narrow(c, nullptr, 0, nullptr, 0, 0, nullptr, nullptr, 0, nullptr, 0, nullptr, 0, c->opts.delta,
                               c->opts.min_sep, c->opts.max_iter, 1, nullptr, nullptr, s, false, 0, nullptr, nullptr,
                               0, false, 1);
  if (rc) return rc;
  int32_t h = CCD_OK;
  CK(cudaMemcpyAsync(&h, &c->ctl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  *status = h;
  return CCD_OK;
}

int ccd_selftest_radix_sort(ccd_ctx *c, int key_bytes, int key_bits, int64_t n, int64_t n_cap, int skip_all,
                            void *keys, uint32_t *vals, int32_t *status, void *stream) {
  if (!c || !status || (key_bytes != 4 && key_bytes != 8) || key_bits < 0 || key_bits > 8 * key_bytes || n < 0 ||
      n_cap < n || n_cap >= (1ll << 32) || (n > 0 && (!keys || !vals)))
    return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t cap = std::max<int64_t>(n_cap, 1);
  const size_t wb = sort_work_bytes(cap);
  char *m = nullptr;
  if (cudaMalloc(&m, 2 * cap * (key_bytes + 4) + wb + 1024) != cudaSuccess) return CCD_ENOMEM;
  void *kb[2] = {m, m + cap * key_bytes};
  uint32_t *vb[2] = {(uint32_t *)(m + 2 * cap * key_bytes), (uint32_t *)(m + 2 * cap * key_bytes) + cap};
  char *wm = m + 2 * cap * (key_bytes + 4);
  wm = (char *)(((uintptr_t)wm + 255) & ~(uintptr_t)255);
  unsigned long long *n_dev = (unsigned long long *)(wm + wb);
  int rc = CCD_OK;
  int32_t h = CCD_OK;
  int cur = 0;
  const unsigned long long un = (unsigned long long)n;
  if (cudaMemsetAsync(wm, 0, wb, s) != cudaSuccess ||
      cudaMemcpyAsync(n_dev, &un, sizeof(un), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      (n > 0 && (cudaMemcpyAsync(kb[0], keys, n * key_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                 cudaMemcpyAsync(vb[0], vals, n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess))) {
    rc = CCD_ECUDA;
  } else {
    k_reset_status<<<1, 1, 0, s>>>(c->ctl);
    const int *sel = nullptr;
    cur = radix_sort(kb, vb, key_bytes, n_cap, sort_work_at(wm), s, &c->ctl->status, key_bits,
                     n_cap > n ? n_dev : nullptr, skip_all ? &sel : nullptr);
    if (sel && (cudaMemcpyAsync(&cur, sel, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                cudaStreamSynchronize(s) != cudaSuccess))
      rc = CCD_ECUDA;
    else if ((n > 0 && (cudaMemcpyAsync(keys, kb[cur], n * key_bytes, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
                   cudaMemcpyAsync(vals, vb[cur], n * 4, cudaMemcpyDeviceToDevice, s) != cudaSuccess)) ||
        cudaMemcpyAsync(&h, &c->ctl->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      rc = CCD_ECUDA;
  }
  cudaStreamSynchronize(s);
  cudaFree(m);
  *status = h;
  return rc;
}

int ccd_get_memory_model(const ccd_opts *o, ccd_memory_model *m) {
  if (!m) return CCD_EINVAL;
  ccd_opts opts;
  ccd_default_opts(&opts);
  if (o) opts = *o;
  // per box, as laid out by ensure_broad: FP32 and FP64 extents, vertex ids,
  // sort keys and values, the sort's look-back states (8 passes x 2 KB per
  // 4096 keys) and the sorted arrays (with the 1-byte tag) for 3 copies per
  // box (strip sweep), the one-list sorted arrays, copy offsets; plus the
  // scene index
  m->bytes_per_box = 24 + 48 + 16 + 3 * (16 + 8) + 3 * 4 + 4 + 3 * (4 + 16 + 16 + 1) + (8 + 8 + 32) + 4 + 4;
  // and the narrow phase's per-primitive set-up record (at most a face's)
  m->bytes_per_box += narrow_prim_words(0, 0, 1) * 8;
  // per pair slot: the pair (8), two candidate slots (16), and the narrow
  // phase's per-query flags (4), counter (8), record (24 words + 33 floats)
  // and scene (4)
  m->bytes_per_pair = 8 + 16 + 4 + 8 + (24 * 8 + 33 * 4) + 4;
  // per scene: statistics, axis and strip layout
  m->bytes_per_scene = 9 * 4 + 6 * 4 + 4 + (int64_t)sizeof(StripParam);
  const int64_t ring = opts.queue_capacity > 0 ? opts.queue_capacity : (1 << 21);
  m->bytes_fixed = ring * (int64_t)sizeof(RingCell) + (int64_t)sizeof(DevCtl) + 64 * 256;
  return CCD_OK;
}

int64_t ccd_pair_capacity_for(const ccd_opts *o, int64_t mem_bytes, int64_t n_boxes, int32_t n_scenes) {
  ccd_memory_model m;
  if (n_boxes < 0 || n_scenes < 0 || ccd_get_memory_model(o, &m) != CCD_OK) return 0;
  const int64_t rest = mem_bytes - m.bytes_fixed - std::max<int64_t>(n_boxes, 1024) * m.bytes_per_box -
                       (int64_t)n_scenes * m.bytes_per_scene;
  return rest > 0 ? rest / m.bytes_per_pair : 0;
}

int ccd_get_status(ccd_ctx *c, ccd_stats *st) {
  if (!c) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  DevCtl h;
  CK(cudaMemcpyAsync(&h, c->ctl, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->last_stream));
  CK(cudaStreamSynchronize(c->last_stream));
  if (st) {
    std::memset(st, 0, sizeof(*st));
    st->n_boxes = c->last_nB;
    st->sweep_axis = h.axis;
    st->n_superset = (int64_t)h.n_superset;
    st->n_vf = (int64_t)h.n_vf;
    st->n_ee = (int64_t)h.n_ee;
    st->n_intervals = (int64_t)h.n_intervals;
    st->n_exported = (int64_t)h.n_exported;
    st->n_donated = (int64_t)h.n_donated;
    st->n_intervals_tail = (int64_t)h.n_intervals_tail;
    st->n_intervals_fp64 = (int64_t)h.n_intervals_fp64;
    st->n_capped = (int64_t)h.n_capped;
    st->queue_peak = (int64_t)h.queue_peak;
    st->device_status = h.status;
    st->n_launches = c->n_launches;
    st->n_box_copies = h.n_copies ? (int64_t)h.n_copies : c->last_nB;
    st->n_ranges = c->last_ranges;
    if (h.t_end > h.t_start && h.t_start) {
      const unsigned long long tx = h.t_exhausted ? h.t_exhausted : h.t_end;
      st->narrow_bulk_ns = (int64_t)(tx - h.t_start);
      st->narrow_tail_ns = (int64_t)(h.t_end - tx);
    }
  }
  return h.status;
}

int ccd_stage_times(ccd_ctx *c, double ms[CCD_NSTAGES]) {
  if (!c || !ms || !c->opts.profile_stages) return CCD_EINVAL;
  CK(cudaSetDevice(c->device));
  CK(cudaStreamSynchronize(c->last_stream));
  for (int k = 0; k < CCD_NSTAGES; ++k) {
    ms[k] = 0.0;
    if (!c->ran[k]) continue;
    float f = 0.f;
    CK(cudaEventElapsedTime(&f, c->ev[2 * k], c->ev[2 * k + 1]));
    ms[k] = f;
  }
  return CCD_OK;
}

const char *ccd_status_str(int s) {
  switch (s) {
    case CCD_OK: return "ok";
    case CCD_EINVAL: return "invalid argument";
    case CCD_ENOMEM: return "device allocation failed";
    case CCD_ETRUNC: return "output list too small (counts hold the sizes needed)";
    case CCD_EQUEUE: return "narrow-phase interval queue overflowed";
    case CCD_ETIMEOUT: return "a bounded device wait gave up; results invalid";
    case CCD_ECUDA: return "CUDA runtime error";
    case CCD_EDEVICE: return "device is not compute capability 10.3";
    default: return "unknown status";
  }
}

}  // extern "C"
