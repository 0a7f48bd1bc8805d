// Kernel interfaces and the device control block shared by the host runtime.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/ccd.h"

namespace ccd {

// Device-resident control block: counters, status and the shared t*.  One
// per context; reset (partially) by the host before each call.
struct DevCtl {
  // broad phase
  unsigned long long n_vf, n_ee, n_superset;
  double var_sum[6];             // sum of centres and squared centres per axis
  int axis;
  int status;                    // CCD_* raised by kernels (first error wins)
  // narrow phase: the words every warp reads or updates sit on their own
  // 128-byte lines, so that atomics on one do not queue behind traffic on
  // another
  alignas(128) unsigned long long q_next;   // next query to hand out
  // ring positions (monotonic; reset only with the ring itself): the head,
  // moved by idle warps taking work, and the tail, moved by warps handing
  // work out, on lines of their own
  alignas(128) unsigned long long q_head;
  alignas(128) unsigned long long q_tail;
  alignas(128) unsigned long long pending;  // units fetched or queued and not finished
  alignas(128) unsigned long long toi_bits; // earliest t* so far, bits of a non-negative double
  alignas(128) unsigned long long n_intervals;
  unsigned long long n_exported, n_capped, queue_peak;
  long long pair_counts[2];      // ccd_step: pairs for the narrow phase (clamped)
  unsigned long long t_start, t_exhausted, t_end;  // %globaltimer stamps of the narrow kernel
  unsigned long long n_donated;  // subtrees passed between lanes of a warp or warps of a block
  unsigned long long n_intervals_tail;  // intervals evaluated after the query list ran out
  unsigned long long n_intervals_fp64;  // intervals the FP32 filter could not decide
  int rerun;                     // zero-TOI rule: 1 when the second pass must run
  unsigned n_left;               // warps of the narrow launch that have left it
  // strip sweep
  unsigned long long n_copies;   // boxes placed in strips (with repeats)
  int strip_fallback;            // 1: the copies did not fit; one cell per scene
  int sup_overflow;              // 1: the candidate buffer of the strip sweep overflowed
  int copy_oversize;             // 1: a box overlaps more cells than its count can hold
  int pad3_;
};

struct RingCell {
  unsigned long long seq;
  unsigned long long w[3];       // numerator | level << 54, for t, u, v
  uint32_t q;
  uint32_t pad;
};

constexpr int kNarrowThreads = 128;
// Claimed queries staged per warp in dynamic shared memory: two buffers of
// kStageQ query records (24 words, 33 floats, scene id each).
constexpr int kStageQ = 16;
static_assert(kStageQ % 4 == 0, "staged records are copied in 16-byte chunks");
constexpr size_t kStageBytes = kStageQ * (24 * 8 + 33 * 4 + 4);
constexpr size_t kNarrowDynSmem = (kNarrowThreads / 32) * 2 * kStageBytes;

struct NarrowArgs {
  DevCtl *ctl;
  const int32_t *vf;             // [n_vf][2]
  const int32_t *ee;             // [n_ee][2]
  int64_t n_vf, n_ee;
  int counts_from_ctl;           // 1: take n_vf, n_ee from ctl->pair_counts
  int64_t ee_end;                // > 0: one shared pair buffer of ee_end pairs, vertex-face
                                 // from the front (vf), edge-edge from the back: the edge-edge
                                 // list is the last n_ee pairs (with counts_from_ctl)
  const double *V0, *V1;         // [3][nV]
  int64_t nV, nE, nF;
  const int32_t *E, *F;
  double *prims;                 // per-primitive set-up records (k_prepare_prims): vertices,
                                 // then edges, then faces; narrow_prim_words(nV, nE, nF) words
  double delta, min_sep;
  long long max_iter;
  int mode;                      // 0 per pair, 1 earliest only, 2 earliest per scene
  int budget;                    // tail phase: every 32 x budget evaluations of a warp, its busy
                                 // lanes hand out their shallowest pending siblings
  int no_zero;                   // zero-TOI rule: intervals with t_lo = 0 are always split
  int only_if_rerun;             // return at once unless ctl->rerun is set
  unsigned long long *toi_vf_bits, *toi_ee_bits;   // mode 0 outputs (bits of doubles)
  uint32_t *qflags;              // [n_vf + n_ee] scratch
  unsigned long long *qiters;    // [n_vf + n_ee] scratch
  RingCell *ring;
  unsigned long long ring_mask;  // capacity - 1
  // batched scenes (mode 2): per-scene earliest time, scene of each query
  int n_scenes;
  const int64_t *voff;
  unsigned long long *toi_scene; // [n_scenes] bits of each scene's t* (+inf initialised)
  int *qsid;                     // [n_vf + n_ee] scene of each query
  unsigned long long *qrec;      // query records: 24 words then 33 floats, x rec_stride
                                 // (NULL: lanes set their queries up themselves)
  int64_t rec_stride;
};

__global__ void k_narrow(NarrowArgs A);         // on query records (A.qrec required)
__global__ void k_narrow_setup(NarrowArgs A);   // lanes set queries up themselves (A.qrec unused)
__global__ void k_prepare_queries(NarrowArgs A);   // needs A.prims from k_prepare_prims
__global__ void k_prepare_prims(NarrowArgs A);
// words of the per-primitive records: 4 per vertex, 10 per edge, 18 per face
constexpr int64_t narrow_prim_words(int64_t nV, int64_t nE, int64_t nF) { return 4 * nV + 10 * nE + 18 * nF; }
__global__ void k_ring_init(RingCell *ring, unsigned long long cap, unsigned long long base);
__global__ void k_nozero_prepare(DevCtl *ctl);
__global__ void k_nozero_finish(DevCtl *ctl);
__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v);
__global__ void k_flags_out(const uint32_t *qflags, int64_t n_vf, int64_t n_ee, uint8_t *flags_vf,
                            uint8_t *flags_ee, DevCtl *ctl);

// ---- broad phase ----
constexpr int kBuildThreads = 256;
constexpr int kOsThreads = 256;                // radix sort: threads per tile
constexpr int kOsItems = 16;                   // keys per thread per tile
constexpr int kOsTile = kOsThreads * kOsItems;
constexpr int kMaxSortPasses = 8;              // 8-bit digits of a 64-bit key

// Cell sweep.  Per scene, the boxes are binned into a grid of cells on the
// two axes other than the sweep axis (a box goes into every cell it
// overlaps) and the sweep runs inside each cell; a pair is reported only in
// the cell where, on each of the two axes, the later of the two minima
// falls, so it is reported once.
constexpr int kMaxCellsSingle = 4095;    // per axis, one scene (24-bit cell index)
constexpr int kMaxCellsBatched = 255;    // per axis, batched scenes (16-bit cell index)
struct StripParam {
  float org[2];                  // smallest box minimum on each cell axis
  float inv_w[2];                // 1 / cell width (0: one cell on that axis)
  int ncell[2];                  // cells on each axis, >= 1
  int axes;                      // sweep axis | first cell axis << 2 | second cell axis << 4
  int pad;
};

// Cell of a coordinate x >= org on cell axis k: monotone non-decreasing in
// x, which is all the reporting rule needs (two boxes that overlap on that
// axis share the cell of the larger of their minima).
__device__ __forceinline__ int strip_of(float x, const StripParam &p, int k) {
  if (p.ncell[k] <= 1) return 0;
  const float t = __fmul_rn(__fsub_rn(x, p.org[k]), p.inv_w[k]);
  return t >= (float)(p.ncell[k] - 1) ? p.ncell[k] - 1 : (t > 0.f ? (int)t : 0);
}

// The same for an FP64 coordinate (the FP64 form bins on FP64 extents).
__device__ __forceinline__ int strip_of64(double x, const StripParam &p, int k) {
  if (p.ncell[k] <= 1) return 0;
  const double t = __dmul_rn(__dsub_rn(x, (double)p.org[k]), (double)p.inv_w[k]);
  return t >= (double)(p.ncell[k] - 1) ? p.ncell[k] - 1 : (t > 0.0 ? (int)t : 0);
}

// Inverse of the ordered-int64 map of a double (f64_ord).
__device__ __forceinline__ double f64_from_ord(long long k) {
  return __longlong_as_double(k >= 0 ? k : (k ^ 0x7FFFFFFFFFFFFFFFll));
}

struct BroadBufs {
  // by box id
  float *lo32, *hi32;            // [3][nB]
  long long *lo64, *hi64;        // [3][nB] ordered FP64 keys
  int4 *vid;                     // [nB] (v0, v1, v2, box id), -1 padded
  // sort (keys are 4 or 8 bytes: single-precision or FP64 form)
  void *keys[2];                 // [nB]
  uint32_t *vals[2];             // [nB]
  // sorted by the minimum on the sweep axis
  float *s_alo, *s_ahi;          // [nB]
  float4 *s_oth;                 // [nB] (lo1, hi1, lo2, hi2)
  int4 *s_vid;                   // [nB]
  uint8_t *s_tag;                // [copies] cell sweep: box kind | first-cell flags << 2
  float *partials;               // [kStatWords * nBuildBlocks]
  // FP64 form: sorted ordered-int64 extents
  long long *s_alo64, *s_ahi64;  // [nB]
  longlong2 *s_oth64;            // [2 * nB]: (lo1, hi1), (lo2, hi2)
  // batched scenes (n_scenes = 0: one scene): scene s owns vertices
  // [voff[s], voff[s+1]), edges [eoff[s], ...), faces [foff[s], ...)
  int n_scenes;
  const int64_t *voff, *eoff, *foff;   // device [n_scenes + 1], starting at 0
  int *bsid;                     // [nB] scene of each box
  float *ssum;                   // [9][n_scenes] sums of centres, squared centres, widths
  uint32_t *smm;                 // [6][n_scenes] ordered keys: min of minima, max of maxima
  int *saxis;                    // [n_scenes] sweep axis per scene
  // strip sweep
  StripParam *sparam;            // [max(1, n_scenes)]
  float strip_factor;            // strip width / mean box width on the strip axis
  int64_t cap_copies;            // capacity of the sorted arrays and sort buffers
  uint32_t *c_local;             // [nB] offset of a box's copies within its block
  unsigned long long *c_blk;     // [nB / kCopyBlock + 1] copies per block, then their prefix
  // FP64 form of the strip sweep (bins and sorts on FP64 extents), [cap_copies] each
  int strips_fp64;               // 1: strips from the FP64 extents
  uint32_t *c_box, *c_seg;       // copy -> box id, strip segment
  uint32_t *s_seg;               // sorted: strip segment
  long long *s_key64, *s_ahi64c; // sorted: ordered FP64 minimum / maximum on the sweep axis
  longlong2 *s_oth64c;           // sorted: [2 per copy] the two other axes
};

constexpr int kStatWords = 15;   // per block: 3 centre sums, 3 squares, 3 widths, 3 min, 3 max
constexpr int kCopyBlock = 1024; // boxes per block of the copy count

// Scene of a primitive (batched scenes): largest s with off[s] <= id.
__device__ __forceinline__ int scene_of(const int64_t *off, int n_scenes, int64_t id) {
  int lo = 0, hi = n_scenes - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= id) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__global__ void k_build_boxes(int64_t nV, int64_t nE, int64_t nF, const double *V0, const double *V1,
                              const int32_t *E, const int32_t *F, BroadBufs B);
__global__ void k_axis_select(const float *partials, int nblocks, int64_t nB, DevCtl *ctl, StripParam *sp,
                              float strip_factor);
__global__ void k_count_copies(int64_t nB, BroadBufs B, DevCtl *ctl);
__global__ void k_scan_copies(int nblk, int64_t nB, BroadBufs B, DevCtl *ctl);
__global__ void k_expand_copies(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys,
                                uint32_t *vals);
__global__ void k_gather_copies(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys0,
                                const unsigned long long *keys1, const uint32_t *perm0, const uint32_t *perm1,
                                const int *sel);
__global__ void k_make_keys(int64_t nB, const float *lo32, const DevCtl *ctl, uint32_t *keys, uint32_t *vals);
__global__ void k_axis_select_scenes(BroadBufs B);
__global__ void k_make_keys_scenes(int64_t nB, BroadBufs B, unsigned long long *keys, uint32_t *vals);
__global__ void k_make_keys64(int64_t nB, const long long *lo64, const DevCtl *ctl, unsigned long long *keys,
                              uint32_t *vals);
// Stable LSD radix sort of (key, value) pairs, 8 bits per pass, on stream s;
// keys[0]/vals[0] hold the input; returns the index (0 or 1) of the buffers
// holding the sorted output.  key_bytes = 4 or 8; only the low key_bits (0:
// all) are sorted on.  Launches one counting kernel and one kernel per pass.
// n_dev (optional): device count, read by the kernels, of the keys to sort
// (at most n; grids are sized for n).  W holds at least sort_work_bytes(n)
// bytes, zeroed once when allocated.  A look-back wait that runs out raises
// CCD_ETIMEOUT in *status.  Passes of a digit that every key shares are
// skipped two at a time, so that the result lands where running every pass
// puts it -- or, with result_sel, all of them: *result_sel is then set to
// a device int naming the result's buffers (0 or 1) and the return value
// means nothing.
struct SortPlan {
  unsigned long long n;                         // keys sorted
  uint32_t blocks_done;                         // counting blocks finished
  uint32_t tiles_next[kMaxSortPasses];          // next tile of each pass
  int run[kMaxSortPasses];                      // the pass moves data
  int in[kMaxSortPasses + 1];                   // buffer pass p reads; in[passes]: the result
  uint32_t base[kMaxSortPasses][256];           // first output position of each digit
};
struct SortWork {
  SortPlan *plan;
  uint32_t *ghist;                              // [kMaxSortPasses][256], zero between sorts
  unsigned long long *states;                   // [passes][tiles][256] look-back states
};
int64_t sort_tiles(int64_t n);
inline size_t sort_work_bytes(int64_t n) {
  return sizeof(SortPlan) + kMaxSortPasses * 256 * sizeof(uint32_t) +
         (size_t)kMaxSortPasses * (size_t)sort_tiles(n) * 256 * sizeof(unsigned long long) + 512;
}
inline SortWork sort_work_at(void *base) {
  char *m = (char *)base;
  SortWork W;
  W.plan = (SortPlan *)m;
  W.ghist = (uint32_t *)(m + ((sizeof(SortPlan) + 255) & ~size_t(255)));
  W.states = (unsigned long long *)((char *)W.ghist + kMaxSortPasses * 256 * sizeof(uint32_t));
  return W;
}
int radix_sort(void *keys[2], uint32_t *vals[2], int key_bytes, int64_t n, const SortWork &W, cudaStream_t s,
               int *status, int key_bits = 0, const unsigned long long *n_dev = nullptr,
               const int **result_sel = nullptr);
__global__ void k_gather_sorted(int64_t nB, const uint32_t *perm, const DevCtl *ctl, BroadBufs B);
__global__ void k_gather_sorted64(int64_t nB, const uint32_t *perm, const DevCtl *ctl, BroadBufs B);

struct SweepArgs {
  int64_t nB, nV, nE;
  int n_scenes;                  // 0: one scene
  const int64_t *voff, *eoff, *foff;
  const int *bsid;
  const float *s_alo, *s_ahi;
  const float4 *s_oth;
  const long long *s_alo64, *s_ahi64;
  const longlong2 *s_oth64;
  const int4 *s_vid;
  const uint8_t *s_tag;          // cell sweep: kind (0 vertex, 1 edge, 2 face) | first-cell flags << 2
  const long long *lo64, *hi64;  // [3][nB] by box id
  int32_t *vf_out, *ee_out;
  int64_t vf_cap, ee_cap;
  int ee_rev;                    // 1: edge-edge pair k goes to slot ee_cap - 1 - k (shared buffer)
  DevCtl *ctl;
  // strip sweep: sorted keys (strip segment << 32 | minimum on the sweep
  // axis) and the number of box copies, both on the device
  const unsigned long long *s_key;
  const unsigned long long *n_dev;
  // strip sweep: single-precision candidates (vertex-face: bit 31 of x set),
  // tested against the FP64 extents by k_exact_filter
  uint2 *sup;
  int64_t sup_cap;
  // cell sweeps: sorted copies [i_begin, i_end) start ranges (the paper's
  // batching: a range's pairs fit the buffers; ranges read past their end)
  int64_t i_begin, i_end;
  // FP64 cell sweep
  const uint32_t *s_seg;
  const long long *s_key64, *s_ahi64c;
  const longlong2 *s_oth64c;
};
__global__ void k_sweep(SweepArgs A);
__global__ void k_sweep_strips(SweepArgs A);
__global__ void k_sweep_strips64(SweepArgs A);
__global__ void k_expand_copies64(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys,
                                  uint32_t *vals);
__global__ void k_gather_seg(int64_t cap, const DevCtl *ctl, const uint32_t *perm, const uint32_t *seg,
                             uint32_t *out);
__global__ void k_gather_copies64(int64_t nB, BroadBufs B, const DevCtl *ctl, const uint32_t *perm);
__global__ void k_exact_filter(SweepArgs A);
__global__ void k_reset_sweep(DevCtl *ctl);
__global__ void k_sweep_tiled(SweepArgs A);
__global__ void k_sweep64(SweepArgs A);

}  // namespace ccd
