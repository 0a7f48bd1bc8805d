// Broad phase: boxes (Section "Construction of the Boxes") and
// sweep-and-prune (Section "Broad-Phase", Algorithm 2).
//
//   k_build_boxes    one thread per box: FP64 extents over t = 0 and t = 1 of
//                    the box's 1-3 vertices, single-precision box by directed
//                    rounding (round-down / round-up, the same float the
//                    paper's round-to-nearest-then-nextafterf rule gives),
//                    order-preserving integer keys of the FP64 extents for the
//                    exact test, and per-block statistics (centre variance,
//                    mean widths, extents).
//   k_axis_select    sweep axis (largest centre variance) and the cell layout
//                    on the two other axes (both affect speed only).
//   k_*_copies       one copy of each box per cell it overlaps, keyed by
//                    (cell, ordered bits of the minimum on the sweep axis).
//   k_sort_*         stable LSD radix sort of the keys, 8 bits per pass, one
//                    kernel per pass (decoupled look-back across tiles).
//   k_sweep_strips   the cell sweep (default): one thread per sorted copy
//                    walks its range in its cell; a pair is reported in one
//                    cell only; candidates go to a list for the exact filter.
//   k_exact_filter   the FP64 box test, vertex-face / edge-edge split and
//                    compaction of the candidate list.
//   k_sweep          Algorithm 2 as printed (sweep_kernel = 1): one warp per
//                    sorted box i, lanes test i against j = i+1, i+2, ... while
//                    min_a(j) <= max_a(i), with the two other axes, the
//                    vertex-face / edge-edge rule, the shared-vertex filter and
//                    the exact FP64 box test fused.
//   k_sweep_tiled    one sorted list, tiles staged in shared memory
//                    (sweep_kernel = 2).

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

namespace ccd {

__global__ void __launch_bounds__(kBuildThreads)
k_build_boxes(int64_t nV, int64_t nE, int64_t nF, const double *__restrict__ V0,
              const double *__restrict__ V1, const int32_t *__restrict__ E,
              const int32_t *__restrict__ F, BroadBufs B) {
  const int64_t nB = nV + nE + nF;
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  // statistics for the axis choice and the strip layout: centre, squared
  // centre, width, minimum and maximum per axis (neutral values for no box)
  float c[3] = {0.f, 0.f, 0.f}, wd[3] = {0.f, 0.f, 0.f};
  float mn[3] = {__int_as_float(0x7F800000), __int_as_float(0x7F800000), __int_as_float(0x7F800000)};
  float mx[3] = {-__int_as_float(0x7F800000), -__int_as_float(0x7F800000), -__int_as_float(0x7F800000)};
  if (b < nB) {
    int ids[3] = {-1, -1, -1};
    int k;
    if (b < nV) {
      ids[0] = (int)b;
      k = 1;
    } else if (b < nV + nE) {
      ids[0] = __ldg(&E[2 * (b - nV)]);
      ids[1] = __ldg(&E[2 * (b - nV) + 1]);
      k = 2;
    } else {
      int64_t f = b - nV - nE;
      ids[0] = __ldg(&F[3 * f]);
      ids[1] = __ldg(&F[3 * f + 1]);
      ids[2] = __ldg(&F[3 * f + 2]);
      k = 3;
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      double lo = __ldg(&V0[a * nV + ids[0]]), hi = lo;
      double x = __ldg(&V1[a * nV + ids[0]]);
      lo = dmin_int(lo, x);
      hi = dmax_int(hi, x);
      for (int i = 1; i < k; ++i) {
        double y0 = __ldg(&V0[a * nV + ids[i]]);
        double y1 = __ldg(&V1[a * nV + ids[i]]);
        lo = dmin_int(dmin_int(lo, y0), y1);
        hi = dmax_int(dmax_int(hi, y0), y1);
      }
      float lo32 = __double2float_rd(lo);
      float hi32 = __double2float_ru(hi);
      B.lo32[a * nB + b] = lo32;
      B.hi32[a * nB + b] = hi32;
      B.lo64[a * nB + b] = f64_ord(lo);
      B.hi64[a * nB + b] = f64_ord(hi);
      c[a] = 0.5f * (lo32 + hi32);
      wd[a] = hi32 - lo32;
      mn[a] = lo32;
      mx[a] = hi32;
    }
    B.vid[b] = make_int4(ids[0], ids[1], ids[2], (int)b);
  }
  const float v[9] = {c[0], c[1], c[2], c[0] * c[0], c[1] * c[1], c[2] * c[2], wd[0], wd[1], wd[2]};
  if (B.n_scenes > 0) {
    // batched scenes: the box's scene, and the statistics per scene (one
    // atomic per warp and word when the warp's boxes share a scene, which is
    // the usual case)
    int sid = 0;
    if (b < nB)
      sid = b < nV ? scene_of(B.voff, B.n_scenes, b)
                   : (b < nV + nE ? scene_of(B.eoff, B.n_scenes, b - nV) : scene_of(B.foff, B.n_scenes, b - nV - nE));
    if (b < nB) B.bsid[b] = sid;
    uint32_t kmn[3], kmx[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      kmn[a] = f32_sort_key(mn[a]);
      kmx[a] = f32_sort_key(mx[a]);
    }
    const int ns = B.n_scenes;
    const unsigned valid = __ballot_sync(0xFFFFFFFFu, b < nB);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, b < nB ? sid : -1);
    if (peers == 0xFFFFFFFFu && valid == 0xFFFFFFFFu) {
      float s9[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        s9[i] = v[i];
        for (int o = 16; o; o >>= 1) s9[i] += __shfl_xor_sync(0xFFFFFFFFu, s9[i], o);
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        kmn[a] = __reduce_min_sync(0xFFFFFFFFu, kmn[a]);
        kmx[a] = __reduce_max_sync(0xFFFFFFFFu, kmx[a]);
      }
      if ((threadIdx.x & 31) == 0) {
        for (int i = 0; i < 9; ++i) atomicAdd(&B.ssum[i * ns + sid], s9[i]);
        for (int a = 0; a < 3; ++a) {
          atomicMin(&B.smm[a * ns + sid], kmn[a]);
          atomicMax(&B.smm[(3 + a) * ns + sid], kmx[a]);
        }
      }
    } else if (b < nB) {
      for (int i = 0; i < 9; ++i) atomicAdd(&B.ssum[i * ns + sid], v[i]);
      for (int a = 0; a < 3; ++a) {
        atomicMin(&B.smm[a * ns + sid], kmn[a]);
        atomicMax(&B.smm[(3 + a) * ns + sid], kmx[a]);
      }
    }
    return;
  }
  // per-block statistics
  float st[kStatWords];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    st[i] = v[i];
    for (int o = 16; o; o >>= 1) st[i] += __shfl_xor_sync(0xFFFFFFFFu, st[i], o);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    st[9 + a] = mn[a];
    st[12 + a] = mx[a];
    for (int o = 16; o; o >>= 1) {
      st[9 + a] = fminf(st[9 + a], __shfl_xor_sync(0xFFFFFFFFu, st[9 + a], o));
      st[12 + a] = fmaxf(st[12 + a], __shfl_xor_sync(0xFFFFFFFFu, st[12 + a], o));
    }
  }
  __shared__ float red[kBuildThreads / 32][kStatWords];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < kStatWords; ++i) red[w][i] = st[i];
  __syncthreads();
  if (threadIdx.x < kStatWords) {
    const int i = threadIdx.x;
    float t = red[0][i];
    for (int j = 1; j < kBuildThreads / 32; ++j)
      t = i < 9 ? t + red[j][i] : (i < 12 ? fminf(t, red[j][i]) : fmaxf(t, red[j][i]));
    B.partials[kStatWords * blockIdx.x + i] = t;
  }
}

// Cell layout of one scene from its statistics: on each of the two axes
// other than the sweep axis, cells strip_factor mean box widths wide (at
// most max_cells of them).
__device__ StripParam make_strip_param(int a, int c0, int c1, double n, const double wsum[2], const float org[2],
                                       const float top[2], float strip_factor, int max_cells) {
  StripParam p;
  p.axes = a | (c0 << 2) | (c1 << 4);
  p.pad = 0;
  for (int k = 0; k < 2; ++k) {
    p.org[k] = 0.f;
    p.inv_w[k] = 0.f;
    p.ncell[k] = 1;
    const double range = (double)top[k] - (double)org[k];
    const double mw = n > 0 ? wsum[k] / n : 0.0;
    const double w = fmax((double)strip_factor * mw, range / max_cells * (1.0 + 1.0 / 1024));
    if (!(range > 0) || !(w > 0) || !isfinite(range) || !isfinite(w)) continue;
    const float inv = (float)(1.0 / w);
    if (!(inv > 0.f) || !isfinite(inv)) continue;
    p.org[k] = org[k];
    p.inv_w[k] = inv;
    p.ncell[k] = (int)fmin((double)max_cells, floor(range * (double)inv) + 1.0);
    if (p.ncell[k] < 1) p.ncell[k] = 1;
  }
  // a thin second axis (fewer than 8 cells) is not binned: its copies would
  // cost more than the comparisons they save
  if (p.ncell[1] < 8) {
    p.ncell[1] = 1;
    p.inv_w[1] = 0.f;
    p.org[1] = 0.f;
  }
  return p;
}

__device__ __forceinline__ void pick_axes(const double var[3], int &a, int &a1) {
  a = 0;
  for (int k = 1; k < 3; ++k)
    if (var[k] > var[a]) a = k;
  a1 = a == 0 ? 1 : 0;
  for (int k = 0; k < 3; ++k)
    if (k != a && var[k] > var[a1]) a1 = k;
}

// Float-float sums (a float and its rounding error) for the statistics: the
// reduction runs on the FP32 pipe (this GPU's FP64 pipe is narrow), with
// about twice float precision, ample for an axis choice and a cell size.
struct FF {
  float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF x, float yh, float yl) {
  const float s = x.hi + yh;
  const float bb = s - x.hi;
  float e = (x.hi - (s - bb)) + (yh - bb);   // exact error of s (two-sum)
  e += x.lo + yl;
  const float h = s + e;
  return FF{h, e - (h - s)};
}

__global__ void k_axis_select(const float *partials, int nblocks, int64_t nB, DevCtl *ctl, StripParam *sp,
                              float strip_factor) {
  __shared__ float acc[24][32];   // per warp: 9 sums (high, low parts), 3 minima, 3 maxima
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  FF s[9];
  float mn[3], mx[3];
#pragma unroll
  for (int j = 0; j < 9; ++j) s[j] = FF{0.f, 0.f};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    mn[a] = __int_as_float(0x7F800000);
    mx[a] = -__int_as_float(0x7F800000);
  }
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
#pragma unroll
    for (int j = 0; j < 9; ++j) s[j] = ff_add(s[j], partials[kStatWords * i + j], 0.f);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = fminf(mn[a], partials[kStatWords * i + 9 + a]);
      mx[a] = fmaxf(mx[a], partials[kStatWords * i + 12 + a]);
    }
  }
  // within each warp, then across the warps (warp 0)
  for (int round = 0; round < 2; ++round) {
#pragma unroll
    for (int o = 16; o; o >>= 1) {
#pragma unroll
      for (int j = 0; j < 9; ++j)
        s[j] = ff_add(s[j], __shfl_xor_sync(0xFFFFFFFFu, s[j].hi, o), __shfl_xor_sync(0xFFFFFFFFu, s[j].lo, o));
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        mn[a] = fminf(mn[a], __shfl_xor_sync(0xFFFFFFFFu, mn[a], o));
        mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xFFFFFFFFu, mx[a], o));
      }
    }
    if (round == 1) break;
    if (lane == 0) {
#pragma unroll
      for (int j = 0; j < 9; ++j) {
        acc[j][w] = s[j].hi;
        acc[9 + j][w] = s[j].lo;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        acc[18 + a][w] = mn[a];
        acc[21 + a][w] = mx[a];
      }
    }
    __syncthreads();
    if (w != 0) return;
    const bool have = lane < (int)(blockDim.x >> 5);
#pragma unroll
    for (int j = 0; j < 9; ++j) s[j] = have ? FF{acc[j][lane], acc[9 + j][lane]} : FF{0.f, 0.f};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      mn[a] = have ? acc[18 + a][lane] : __int_as_float(0x7F800000);
      mx[a] = have ? acc[21 + a][lane] : -__int_as_float(0x7F800000);
    }
  }
  if (threadIdx.x == 0) {
    double t[kStatWords];
#pragma unroll
    for (int j = 0; j < 9; ++j) t[j] = (double)s[j].hi + (double)s[j].lo;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      t[9 + a] = mn[a];
      t[12 + a] = mx[a];
    }
    double inv = nB > 0 ? 1.0 / (double)nB : 0.0;
    double var[3];
    for (int a = 0; a < 3; ++a) {
      double mean = t[a] * inv;
      var[a] = t[3 + a] * inv - mean * mean;
      ctl->var_sum[a] = t[a];
      ctl->var_sum[3 + a] = t[3 + a];
    }
    int a, b;
    pick_axes(var, a, b);
    ctl->axis = a;
    const int c = 3 - a - b;
    const double ws[2] = {t[6 + b], t[6 + c]};
    const float lo[2] = {(float)t[9 + b], (float)t[9 + c]}, hi[2] = {(float)t[12 + b], (float)t[12 + c]};
    sp[0] = make_strip_param(a, b, c, (double)nB, ws, lo, hi, strip_factor, kMaxCellsSingle);
  }
}

__global__ void k_make_keys(int64_t nB, const float *lo32, const DevCtl *ctl, uint32_t *keys, uint32_t *vals) {
  const int a = ctl->axis;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nB; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = f32_sort_key(lo32[a * nB + i]);
    vals[i] = (uint32_t)i;
  }
}

// Batched scenes: axis of largest centre variance and strip layout per scene.
__device__ __forceinline__ float f32_from_sort_key(uint32_t k) {
  return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

__global__ void k_axis_select_scenes(BroadBufs B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.n_scenes) return;
  const int ns = B.n_scenes;
  const double n = (double)((B.voff[s + 1] - B.voff[s]) + (B.eoff[s + 1] - B.eoff[s]) + (B.foff[s + 1] - B.foff[s]));
  const double inv = n > 0 ? 1.0 / n : 0.0;
  double var[3];
  for (int a = 0; a < 3; ++a) {
    const double mean = (double)B.ssum[a * ns + s] * inv;
    var[a] = (double)B.ssum[(3 + a) * ns + s] * inv - mean * mean;
  }
  int a, b;
  pick_axes(var, a, b);
  B.saxis[s] = a;
  const int c = 3 - a - b;
  double ws[2] = {0.0, 0.0};
  float lo[2] = {0.f, 0.f}, hi[2] = {0.f, 0.f};
  if (n > 0) {
    ws[0] = (double)B.ssum[(6 + b) * ns + s];
    ws[1] = (double)B.ssum[(6 + c) * ns + s];
    lo[0] = f32_from_sort_key(B.smm[b * ns + s]);
    lo[1] = f32_from_sort_key(B.smm[c * ns + s]);
    hi[0] = f32_from_sort_key(B.smm[(3 + b) * ns + s]);
    hi[1] = f32_from_sort_key(B.smm[(3 + c) * ns + s]);
  }
  B.sparam[s] = make_strip_param(a, b, c, n, ws, lo, hi, B.strip_factor, kMaxCellsBatched);
}

// Batched scenes: key = scene << 32 | ordered bits of the minimum on the
// scene's axis, so that every scene is one contiguous, sorted run.
__global__ void k_make_keys_scenes(int64_t nB, BroadBufs B, unsigned long long *keys, uint32_t *vals) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nB; i += (int64_t)gridDim.x * blockDim.x) {
    const int s = B.bsid[i];
    const int a = B.saxis[s];
    keys[i] = ((unsigned long long)s << 32) | f32_sort_key(B.lo32[a * nB + i]);
    vals[i] = (uint32_t)i;
  }
}

// FP64 form: the ordered int64 extent with its sign bit flipped is an
// unsigned key in numeric order.
__global__ void k_make_keys64(int64_t nB, const long long *lo64, const DevCtl *ctl, unsigned long long *keys,
                              uint32_t *vals) {
  const int a = ctl->axis;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nB; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = (unsigned long long)lo64[a * nB + i] ^ 0x8000000000000000ull;
    vals[i] = (uint32_t)i;
  }
}

// ---- radix sort: one kernel per 8-bit digit, decoupled look-back ----------
//
// k_sort_hist reads the keys once and counts every digit of every pass (the
// global digit totals do not depend on the order), clears the look-back
// states and, in its last block, turns the totals into each pass's digit
// bases.  A pass whose digit is the same for every key would leave the order
// as it is; such passes are skipped two at a time, so that the result always
// lands in the buffers that running every pass would give.  Each k_sort_pass
// block takes the next tile (an atomic counter, so that every earlier tile
// belongs to a block that is already running), ranks its keys stably (warps
// in index order; within a warp, the lanes of equal digit from 8 ballots),
// publishes its per-digit counts, adds up the counts of the tiles before it
// by walking back (16 tiles per round trip) until a tile that has published
// its inclusive prefix, publishes its own prefix and scatters.  The
// walk-back waits are bounded: a wait that runs out raises CCD_ETIMEOUT and
// the scatter stays within the output.

constexpr unsigned long long kAggFlag = 1ull << 62, kPrefixFlag = 2ull << 62;
constexpr unsigned long long kStateValue = (1ull << 62) - 1;
constexpr unsigned kLookbackSpins = 1u << 21;
constexpr int kLookbackWindow = 16;
constexpr int kOsWarps = kOsThreads / 32;

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Lanes of the warp whose 8-bit digit equals this lane's (lanes outside
// `valid` excluded): eight ballots, one per bit.
__device__ __forceinline__ unsigned same_digit_lanes(uint32_t d, unsigned valid) {
  unsigned peers = valid;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const unsigned bb = __ballot_sync(0xFFFFFFFFu, (d >> b) & 1u);
    peers &= ((d >> b) & 1u) ? bb : ~bb;
  }
  return peers;
}

template <typename K>
__global__ void __launch_bounds__(kOsThreads)
k_sort_hist(const K *__restrict__ keys, int64_t n, const unsigned long long *n_dev, int passes, int pair_skip,
            SortWork W) {
  __shared__ uint32_t h[kMaxSortPasses][256];
  __shared__ uint32_t wsum[kOsWarps];
  __shared__ int last;
  __shared__ int constant[kMaxSortPasses];
  if (n_dev) n = min(n, (int64_t)*n_dev);
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int p = 0; p < passes; ++p) {
    W.states[((int64_t)p * gridDim.x + blockIdx.x) * 256 + tid] = 0;   // this tile's look-back states
    h[p][tid] = 0;
  }
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kOsTile;
  if (base < n) {
#pragma unroll 4
    for (int r = 0; r < kOsItems; ++r) {
      const int64_t i = base + r * kOsThreads + tid;
      const bool ok = i < n;
      const K k = ok ? keys[i] : K(0);
      const unsigned valid = __ballot_sync(0xFFFFFFFFu, ok);
      for (int p = 0; p < passes; ++p) {
        // a digit that every valid lane of the warp shares (the common case
        // for the high digits) takes one shared-memory atomic, others one each
        const uint32_t d = (uint32_t)(k >> (8 * p)) & 0xFFu;
        const uint32_t lo = __reduce_min_sync(0xFFFFFFFFu, ok ? d : 0xFFu);
        const uint32_t hi = __reduce_max_sync(0xFFFFFFFFu, ok ? d : 0u);
        if (lo == hi) {
          if (lane == 0 && valid) atomicAdd(&h[p][lo], (uint32_t)__popc(valid));
        } else if (ok) {
          atomicAdd(&h[p][d], 1u);
        }
      }
    }
  }
  __syncthreads();
  for (int p = 0; p < passes; ++p)
    if (h[p][tid]) atomicAdd(&W.ghist[p * 256 + tid], h[p][tid]);
  __threadfence();
  __syncthreads();
  if (tid == 0) last = atomicAdd(&W.plan->blocks_done, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  // the last block: digit bases per pass (exclusive prefix of the totals)
  __threadfence();
  SortPlan *P = W.plan;
  for (int p = 0; p < passes; ++p) {
    const uint32_t v = atomicExch(&W.ghist[p * 256 + tid], 0u);   // read, and clear for the next sort
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    if (tid == 0) constant[p] = 0;
    __syncthreads();
    uint32_t before = 0;
    for (int j = 0; j < w; ++j) before += wsum[j];
    P->base[p][tid] = before + x - v;
    if ((int64_t)v == n) constant[p] = 1;
    __syncthreads();
  }
  if (tid == 0) {
    int nskip = 0, skip_last = -1;
    for (int p = 0; p < passes; ++p) {
      P->run[p] = !constant[p];
      if (constant[p]) {
        ++nskip;
        skip_last = p;
      }
    }
    if (pair_skip && (nskip & 1)) P->run[skip_last] = 1;   // in pairs: the result stays where every pass puts it
    P->in[0] = 0;
    for (int p = 0; p < passes; ++p) {
      P->in[p + 1] = P->in[p] ^ P->run[p];
      P->tiles_next[p] = 0;
    }
    P->n = (unsigned long long)n;
    P->blocks_done = 0;
  }
}

template <typename K>
__global__ void __launch_bounds__(kOsThreads)
k_sort_pass(K *__restrict__ k0, K *__restrict__ k1, uint32_t *__restrict__ v0, uint32_t *__restrict__ v1, int pass,
            SortWork W, int *status) {
  const SortPlan *P = W.plan;
  if (!P->run[pass]) return;
  __shared__ uint32_t wh[kOsWarps][256];   // per warp and digit: count, then the warp's offset in the tile
  __shared__ uint32_t s_pos[256];          // output position of the tile's first key of each digit
  __shared__ uint32_t s_tile;
  __shared__ int s_bad;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) {
    s_tile = atomicAdd(&W.plan->tiles_next[pass], 1u);
    s_bad = 0;
  }
#pragma unroll
  for (int j = 0; j < kOsWarps; ++j) wh[j][tid] = 0;
  __syncthreads();
  const int64_t n = (int64_t)P->n;
  const int64_t tile = s_tile;
  if (tile * kOsTile >= n) return;   // (uniform) beyond the keys
  const int in = P->in[pass];
  const K *kin = in ? k1 : k0;
  K *kout = in ? k0 : k1;
  const uint32_t *vin = in ? v1 : v0;
  uint32_t *vout = in ? v0 : v1;
  const int shift = 8 * pass;
  const int64_t wb = tile * kOsTile + (int64_t)w * (kOsItems * 32);   // the warp's keys, in index order
  K key[kOsItems];
  uint32_t val[kOsItems], off[kOsItems];
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) {
    const int64_t i = wb + r * 32 + lane;
    key[r] = i < n ? kin[i] : K(0);
    val[r] = i < n ? vin[i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) {
    const bool ok = wb + r * 32 + lane < n;
    const uint32_t d = (uint32_t)(key[r] >> shift) & 0xFFu;
    const unsigned peers = same_digit_lanes(d, __ballot_sync(0xFFFFFFFFu, ok));
    const uint32_t before = ok ? wh[w][d] : 0u;
    __syncwarp();
    if (ok && lane == __ffs(peers) - 1) wh[w][d] = before + __popc(peers);
    __syncwarp();
    off[r] = before + __popc(peers & ((1u << lane) - 1u));
  }
  __syncthreads();
  // thread tid handles digit tid: offsets of the warps within the tile
  uint32_t cnt = 0;
#pragma unroll
  for (int j = 0; j < kOsWarps; ++j) {
    const uint32_t c = wh[j][tid];
    wh[j][tid] = cnt;
    cnt += c;
  }
  unsigned long long *st = W.states + (int64_t)pass * gridDim.x * 256;
  unsigned long long excl = 0;
  if (tile == 0) {
    st_relaxed_u64(&st[tid], kPrefixFlag | cnt);
  } else {
    st_relaxed_u64(&st[tile * 256 + tid], kAggFlag | cnt);
    // walk back kLookbackWindow tiles per round trip: add their counts up to
    // the nearest tile with an inclusive prefix; a tile that has published
    // nothing yet is read again (from there) on the next round
    int64_t t = tile - 1;
    unsigned spins = 0;
    while (true) {
      unsigned long long v[kLookbackWindow];
#pragma unroll
      for (int j = 0; j < kLookbackWindow; ++j) v[j] = t - j >= 0 ? ld_relaxed_u64(&st[(t - j) * 256 + tid]) : 0ull;
      int used = 0;
      bool done = false, wait = false;
#pragma unroll
      for (int j = 0; j < kLookbackWindow; ++j) {
        if (done || wait) continue;
        if ((v[j] >> 62) == 0 || t - j < 0) {   // (tile 0 always publishes a prefix: t - j >= 0 here)
          wait = true;
          continue;
        }
        excl += v[j] & kStateValue;
        done = (v[j] & kPrefixFlag) != 0;
        used = j + 1;
      }
      if (done) break;
      t -= used;
      if (wait && used == 0 && ++spins > kLookbackSpins) {   // (a tile before this one never published)
        s_bad = 1;
        break;
      }
    }
    st_relaxed_u64(&st[tile * 256 + tid], kPrefixFlag | (excl + cnt));
  }
  s_pos[tid] = P->base[pass][tid] + (uint32_t)excl;
  __syncthreads();
  if (tid == 0 && s_bad) atomicCAS(status, CCD_OK, CCD_ETIMEOUT);
#pragma unroll
  for (int r = 0; r < kOsItems; ++r) {
    if (wb + r * 32 + lane < n) {
      const uint32_t d = (uint32_t)(key[r] >> shift) & 0xFFu;
      const int64_t pos = (int64_t)s_pos[d] + wh[w][d] + off[r];
      if (pos < n) {   // (always, unless a walk-back gave up)
        kout[pos] = key[r];
        vout[pos] = val[r];
      }
    }
  }
}

int64_t sort_tiles(int64_t n) { return std::max<int64_t>(1, (n + kOsTile - 1) / kOsTile); }

template <typename K>
int radix_sort_t(K *keys[2], uint32_t *vals[2], int64_t n, const SortWork &W, cudaStream_t s, int *status,
                 int key_bits, const unsigned long long *n_dev, const int **result_sel) {
  const int64_t ntiles = sort_tiles(n);
  const int bits = key_bits > 0 ? key_bits : (int)(8 * sizeof(K));
  const int passes = (bits + 7) / 8;
  if (result_sel) *result_sel = &W.plan->in[passes];
  k_sort_hist<K><<<(unsigned)ntiles, kOsThreads, 0, s>>>(keys[0], n, n_dev, passes, result_sel ? 0 : 1, W);
  for (int p = 0; p < passes; ++p)
    k_sort_pass<K><<<(unsigned)ntiles, kOsThreads, 0, s>>>(keys[0], keys[1], vals[0], vals[1], p, W, status);
  return passes & 1;
}

int radix_sort(void *keys[2], uint32_t *vals[2], int key_bytes, int64_t n, const SortWork &W, cudaStream_t s,
               int *status, int key_bits, const unsigned long long *n_dev, const int **result_sel) {
  if (key_bytes == 4) {
    uint32_t *k[2] = {(uint32_t *)keys[0], (uint32_t *)keys[1]};
    return radix_sort_t<uint32_t>(k, vals, n, W, s, status, key_bits, n_dev, result_sel);
  }
  unsigned long long *k[2] = {(unsigned long long *)keys[0], (unsigned long long *)keys[1]};
  return radix_sort_t<unsigned long long>(k, vals, n, W, s, status, key_bits, n_dev, result_sel);
}

__global__ void k_gather_sorted64(int64_t nB, const uint32_t *__restrict__ perm, const DevCtl *ctl, BroadBufs B) {
  const int a = ctl->axis, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nB; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = perm[s];
    B.s_alo64[s] = B.lo64[a * nB + b];
    B.s_ahi64[s] = B.hi64[a * nB + b];
    B.s_oth64[2 * s] = make_longlong2(B.lo64[a1 * nB + b], B.hi64[a1 * nB + b]);
    B.s_oth64[2 * s + 1] = make_longlong2(B.lo64[a2 * nB + b], B.hi64[a2 * nB + b]);
    B.s_vid[s] = B.vid[b];
  }
}

__global__ void k_gather_sorted(int64_t nB, const uint32_t *__restrict__ perm, const DevCtl *ctl, BroadBufs B) {
  for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < nB; s += (int64_t)gridDim.x * blockDim.x) {
    int64_t b = perm[s];
    const int a = B.n_scenes > 0 ? B.saxis[B.bsid[b]] : ctl->axis, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    B.s_alo[s] = B.lo32[a * nB + b];
    B.s_ahi[s] = B.hi32[a * nB + b];
    B.s_oth[s] = make_float4(B.lo32[a1 * nB + b], B.hi32[a1 * nB + b], B.lo32[a2 * nB + b], B.hi32[a2 * nB + b]);
    B.s_vid[s] = B.vid[b];
  }
}

// ---- strip layout: copies of boxes per strip -------------------------------

__device__ __forceinline__ int box_scene(const BroadBufs &B, int64_t b) { return B.n_scenes > 0 ? B.bsid[b] : 0; }

// Cells [s0[k], s1[k]] of box b on its scene's two cell axes.
__device__ __forceinline__ void box_cells(const BroadBufs &B, int64_t nB, int64_t b, const StripParam &p, int s0[2],
                                          int s1[2]) {
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = (p.axes >> (2 + 2 * k)) & 3;
    if (B.strips_fp64) {
      s0[k] = strip_of64(f64_from_ord(B.lo64[x * nB + b]), p, k);
      s1[k] = strip_of64(f64_from_ord(B.hi64[x * nB + b]), p, k);
    } else {
      s0[k] = strip_of(B.lo32[x * nB + b], p, k);
      s1[k] = strip_of(B.hi32[x * nB + b], p, k);
    }
  }
}

// A box's copies, capped so that a block's sum fits 32 bits; a box over the
// cap raises copy_oversize (the layout then falls back to one cell).
constexpr uint32_t kMaxCopiesPerBox = 1u << 21;
__device__ __forceinline__ uint32_t cell_count(const int s0[2], const int s1[2], bool &oversize) {
  const unsigned long long c = (unsigned long long)(s1[0] - s0[0] + 1) * (unsigned long long)(s1[1] - s0[1] + 1);
  oversize = c > kMaxCopiesPerBox;
  return oversize ? kMaxCopiesPerBox : (uint32_t)c;
}

// Copies per box and their exclusive prefix within each block of kCopyBlock
// boxes; the block totals go to c_blk.
__global__ void __launch_bounds__(kCopyBlock) k_count_copies(int64_t nB, BroadBufs B, DevCtl *ctl) {
  __shared__ uint32_t wsum[kCopyBlock / 32];
  const int64_t b = (int64_t)blockIdx.x * kCopyBlock + threadIdx.x;
  uint32_t n = 0;
  if (b < nB) {
    const StripParam p = B.sparam[box_scene(B, b)];
    int s0[2], s1[2];
    box_cells(B, nB, b, p, s0, s1);
    bool over;
    n = cell_count(s0, s1, over);
    if (over) ctl->copy_oversize = 1;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  uint32_t x = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  if (w == 0) {
    const uint32_t v = wsum[lane];
    uint32_t z = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
      if (lane >= o) z += y;
    }
    wsum[lane] = z - v;
    if (lane == 31) B.c_blk[blockIdx.x] = z;
  }
  __syncthreads();
  if (b < nB) B.c_local[b] = wsum[w] + x - n;
}

// Exclusive prefix of the block totals (one block); the total number of
// copies, or the fallback to one strip per scene when they do not fit.
__global__ void __launch_bounds__(1024) k_scan_copies(int nblk, int64_t nB, BroadBufs B, DevCtl *ctl) {
  __shared__ unsigned long long wsum[32];
  __shared__ unsigned long long carry;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nblk; base += 1024) {
    const int i = base + tid;
    const unsigned long long v = i < nblk ? B.c_blk[i] : 0ull;
    unsigned long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    unsigned long long before = carry;
    for (int k = 0; k < w; ++k) before += wsum[k];
    if (i < nblk) B.c_blk[i] = before + x - v;
    __syncthreads();
    if (tid == 1023) carry = before + x;
    __syncthreads();
  }
  if (tid == 0) {
    const bool fit = carry <= (unsigned long long)B.cap_copies && ctl->copy_oversize == 0;
    ctl->strip_fallback = fit ? 0 : 1;
    ctl->n_copies = fit ? carry : (unsigned long long)nB;
  }
}

// Sort keys of the copies: (scene << 16 | strip) << 32 | ordered minimum on
// the scene's sweep axis.  Under the fallback every box has one copy, in
// strip 0 of its scene.
__global__ void k_expand_copies(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys,
                                uint32_t *vals) {
  const bool fallback = ctl->strip_fallback != 0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nB; b += (int64_t)gridDim.x * blockDim.x) {
    const int sid = box_scene(B, b);
    const StripParam p = B.sparam[sid];
    const unsigned long long seg = B.n_scenes > 0 ? ((unsigned long long)sid << 16) : 0ull;
    const uint32_t k = f32_sort_key(B.lo32[(p.axes & 3) * nB + b]);
    if (fallback) {
      keys[b] = (seg << 32) | k;
      vals[b] = (uint32_t)b;
      continue;
    }
    int s0[2], s1[2];
    box_cells(B, nB, b, p, s0, s1);
    unsigned long long o = B.c_blk[b / kCopyBlock] + B.c_local[b];
    for (int t = s0[0]; t <= s1[0]; ++t)
      for (int u = s0[1]; u <= s1[1]; ++u, ++o) {
        keys[o] = ((seg | (unsigned)(t * p.ncell[1] + u)) << 32) | k;
        vals[o] = (uint32_t)b;
      }
  }
}

// Copies in sorted order: maximum on the sweep axis, extents on the strip
// axis and the third axis, vertex ids and box id; bit 31 of the box id marks
// the copy in the box's first strip (the reporting rule of the sweep).  The
// sort leaves its result in buffers *sel (read on the device: it skips the
// passes of digits that every key shares); the sorted keys end in keys0.
__global__ void k_gather_copies(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys0,
                                const unsigned long long *keys1, const uint32_t *perm0, const uint32_t *perm1,
                                const int *sel) {
  const int64_t n = (int64_t)ctl->n_copies;
  const bool fallback = ctl->strip_fallback != 0;
  const bool in1 = *sel != 0;
  const uint32_t *perm = in1 ? perm1 : perm0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = perm[i];
    const unsigned long long key = in1 ? keys1[i] : keys0[i];
    if (in1) keys0[i] = key;
    const int sid = B.n_scenes > 0 ? (int)(key >> 48) : 0;
    const uint32_t cell = B.n_scenes > 0 ? (uint32_t)((key >> 32) & 0xFFFFu) : (uint32_t)(key >> 32);
    const StripParam p = B.sparam[sid];
    const int a = p.axes & 3, a1 = (p.axes >> 2) & 3, a2 = (p.axes >> 4) & 3;
    const float lo1 = B.lo32[a1 * nB + b], lo2 = B.lo32[a2 * nB + b];
    B.s_ahi[i] = B.hi32[a * nB + b];
    B.s_oth[i] = make_float4(lo1, B.hi32[a1 * nB + b], lo2, B.hi32[a2 * nB + b]);
    const uint32_t f0 = fallback || (int)(cell / p.ncell[1]) == strip_of(lo1, p, 0);
    const uint32_t f1 = fallback || (int)(cell % p.ncell[1]) == strip_of(lo2, p, 1);
    const int4 v = B.vid[b];
    B.s_vid[i] = make_int4(v.x, v.y, v.z, (int)((uint32_t)b | (f0 << 31) | (f1 << 30)));
    // kind from the padding: a vertex box has one vertex, an edge two, a face three
    B.s_tag[i] = (uint8_t)((v.y >= 0) + (v.z >= 0) + (f1 << 2) + (f0 << 3));
  }
}

// FP64 form of the strip layout.  Copies carry the ordered FP64 minimum on
// the sweep axis (as an unsigned key) and their strip segment; two stable
// radix sorts order them by the key and then by the segment.
__global__ void k_expand_copies64(int64_t nB, BroadBufs B, const DevCtl *ctl, unsigned long long *keys,
                                  uint32_t *vals) {
  const bool fallback = ctl->strip_fallback != 0;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; b < nB; b += (int64_t)gridDim.x * blockDim.x) {
    const int sid = box_scene(B, b);
    const StripParam p = B.sparam[sid];
    const uint32_t seg = B.n_scenes > 0 ? ((uint32_t)sid << 16) : 0u;
    const unsigned long long k = (unsigned long long)B.lo64[(p.axes & 3) * nB + b] ^ 0x8000000000000000ull;
    int s0[2] = {0, 0}, s1[2] = {0, 0};
    int64_t o = b;
    if (!fallback) {
      box_cells(B, nB, b, p, s0, s1);
      o = (int64_t)(B.c_blk[b / kCopyBlock] + B.c_local[b]);
    }
    for (int t = s0[0]; t <= s1[0]; ++t)
      for (int u = s0[1]; u <= s1[1]; ++u, ++o) {
        keys[o] = k;
        vals[o] = (uint32_t)o;
        B.c_box[o] = (uint32_t)b;
        B.c_seg[o] = seg | (uint32_t)(t * p.ncell[1] + u);
      }
  }
}

__global__ void k_gather_seg(int64_t cap, const DevCtl *ctl, const uint32_t *perm, const uint32_t *seg,
                             uint32_t *out) {
  const int64_t n = (int64_t)ctl->n_copies;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = seg[perm[i]];
}

__global__ void k_gather_copies64(int64_t nB, BroadBufs B, const DevCtl *ctl, const uint32_t *perm) {
  const int64_t n = (int64_t)ctl->n_copies;
  const bool fallback = ctl->strip_fallback != 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t c = perm[i];
    const int64_t b = B.c_box[c];
    const uint32_t seg = B.c_seg[c];
    const int sid = B.n_scenes > 0 ? (int)(seg >> 16) : 0;
    const uint32_t cell = B.n_scenes > 0 ? (seg & 0xFFFFu) : seg;
    const StripParam p = B.sparam[sid];
    const int a = p.axes & 3, a1 = (p.axes >> 2) & 3, a2 = (p.axes >> 4) & 3;
    const long long lo1 = B.lo64[a1 * nB + b], lo2 = B.lo64[a2 * nB + b];
    B.s_seg[i] = seg;
    B.s_key64[i] = B.lo64[a * nB + b];
    B.s_ahi64c[i] = B.hi64[a * nB + b];
    B.s_oth64c[2 * i] = make_longlong2(lo1, B.hi64[a1 * nB + b]);
    B.s_oth64c[2 * i + 1] = make_longlong2(lo2, B.hi64[a2 * nB + b]);
    const uint32_t f0 = fallback || (int)(cell / p.ncell[1]) == strip_of64(f64_from_ord(lo1), p, 0);
    const uint32_t f1 = fallback || (int)(cell % p.ncell[1]) == strip_of64(f64_from_ord(lo2), p, 1);
    const int4 v = B.vid[b];
    B.s_vid[i] = make_int4(v.x, v.y, v.z, (int)((uint32_t)b | (f0 << 31) | (f1 << 30)));
  }
}

// ---- sweep ------------------------------------------------------------------

__device__ __forceinline__ int box_kind(int b, int64_t nV, int64_t nE) {
  return b < nV ? 0 : (b < nV + nE ? 1 : 2);   // vertex, edge, face
}

// Vertex-face / edge-edge rule and shared-vertex filter for a pair of boxes
// whose extents overlap; on success writes the canonical pair.
__device__ __forceinline__ bool candidate(const int4 vi, int ki, const int4 vj, int64_t nV, int64_t nE, bool &is_vf,
                                          int &p0, int &p1) {
  const int bi = vi.w, bj = vj.w;
  const int kj = box_kind(bj, nV, nE);
  const bool vfp = (ki == 0 && kj == 2) || (ki == 2 && kj == 0);
  const bool eep = ki == 1 && kj == 1;
  if (!(vfp || eep)) return false;
  // shared vertex (i padded with -1, j with -2: padding never matches)
  const int j0v = vj.x, j1v = vj.y < 0 ? -2 : vj.y, j2v = vj.z < 0 ? -2 : vj.z;
  const int iv[3] = {vi.x, vi.y, vi.z};
  bool share = false;
#pragma unroll
  for (int u = 0; u < 3; ++u) share |= (iv[u] == j0v) | (iv[u] == j1v) | (iv[u] == j2v);
  if (share) return false;
  is_vf = vfp;
  if (vfp) {
    p0 = ki == 0 ? bi : bj;
    p1 = (int)((ki == 2 ? bi : bj) - nV - nE);
  } else {
    const int e1 = (int)(bi - nV), e2 = (int)(bj - nV);
    p0 = min(e1, e2);
    p1 = max(e1, e2);
  }
  return true;
}

__device__ __forceinline__ void emit(const SweepArgs &A, bool is_vf, bool is_ee, int p0, int p1) {
  const unsigned mask = 0xFFFFFFFFu;
  if (__any_sync(mask, is_vf)) {
    unsigned long long at = warp_append(&A.ctl->n_vf, is_vf, mask);
    if (is_vf && (int64_t)at < A.vf_cap) {
      A.vf_out[2 * at] = p0;
      A.vf_out[2 * at + 1] = p1;
    }
  }
  if (__any_sync(mask, is_ee)) {
    unsigned long long at = warp_append(&A.ctl->n_ee, is_ee, mask);
    if (is_ee && (int64_t)at < A.ee_cap) {
      const int64_t k = A.ee_rev ? A.ee_cap - 1 - (int64_t)at : (int64_t)at;
      A.ee_out[2 * k] = p0;
      A.ee_out[2 * k + 1] = p1;
    }
  }
}

__global__ void __launch_bounds__(256) k_sweep(SweepArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nB = A.nB;
  for (int64_t i = warp; i < nB; i += nwarps) {
    const float ahi = A.s_ahi[i];
    const float4 oi = A.s_oth[i];
    const int4 vi = A.s_vid[i];
    const int bi = vi.w;
    const int ki = box_kind(bi, A.nV, A.nE);
    long long ilo[3], ihi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ilo[a] = A.lo64[a * nB + bi];
      ihi[a] = A.hi64[a * nB + bi];
    }
    for (int64_t j0 = i + 1;; j0 += 32) {
      const int64_t j = j0 + lane;
      const float alo = j < nB ? A.s_alo[j] : __int_as_float(0x7F800000);
      const bool in_a = alo <= ahi;
      const unsigned run = __ballot_sync(0xFFFFFFFFu, in_a);
      bool is_vf = false, is_ee = false, sup = false;
      int p0 = 0, p1 = 0;
      if (in_a) {
        const float4 oj = A.s_oth[j];
        if (oj.x <= oi.y && oi.x <= oj.y && oj.z <= oi.w && oi.z <= oj.w) {
          const int4 vj = A.s_vid[j];
          bool vf;
          if (candidate(vi, ki, vj, A.nV, A.nE, vf, p0, p1)) {
            sup = true;
            // exact test on the FP64 extents (ordered integer keys)
            const int bj = vj.w;
            bool ov = true;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
              long long jlo = A.lo64[a * nB + bj], jhi = A.hi64[a * nB + bj];
              ov &= (jlo <= ihi[a]) & (ilo[a] <= jhi);
            }
            is_vf = ov && vf;
            is_ee = ov && !vf;
          }
        }
      }
      const unsigned bs = __ballot_sync(0xFFFFFFFFu, sup);
      if (bs && lane == 0) atomicAdd(&A.ctl->n_superset, (unsigned long long)__popc(bs));
      emit(A, is_vf, is_ee, p0, p1);
      if (run != 0xFFFFFFFFu) break;   // sorted: later boxes start beyond max_a(i)
    }
  }
}

// Tiled sweep (single-precision form).  A block of 128 threads owns 256
// consecutive sorted boxes, two per thread, and walks the union of their
// sweep ranges in tiles of kTJ boxes staged in shared memory.  At every step
// all lanes test their two boxes against the same box j, so the shared-memory
// reads are broadcasts serving two tests each; the order test j > i is needed
// only while the tile overlaps the block's own boxes; one warp vote covers
// 4 j x 2 boxes.  Tests beyond a box's range fail by themselves (sorted
// minima exceed its maximum).  Survivors of the three single-precision axes
// go through the candidate rule and the exact FP64 test.
constexpr int kSweepThreads = 128;
constexpr int kTI = 2 * kSweepThreads;
constexpr int kTJ = 256;

__device__ __forceinline__ void sweep_hit(const SweepArgs &A, bool hit, const int4 vi, int ki, const int4 vj,
                                          int64_t nB) {
  bool is_vf = false, is_ee = false, sup = false;
  int p0 = 0, p1 = 0;
  if (hit) {
    bool vf;
    if (candidate(vi, ki, vj, A.nV, A.nE, vf, p0, p1)) {
      sup = true;
      bool ov = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const long long ilo = A.lo64[a * nB + vi.w], ihi = A.hi64[a * nB + vi.w];
        const long long jlo = A.lo64[a * nB + vj.w], jhi = A.hi64[a * nB + vj.w];
        ov &= (jlo <= ihi) & (ilo <= jhi);
      }
      is_vf = ov && vf;
      is_ee = ov && !vf;
    }
  }
  const unsigned bs = __ballot_sync(0xFFFFFFFFu, sup);
  if (bs && (threadIdx.x & 31) == 0) atomicAdd(&A.ctl->n_superset, (unsigned long long)__popc(bs));
  emit(A, is_vf, is_ee, p0, p1);
}

__global__ void __launch_bounds__(kSweepThreads) k_sweep_tiled(SweepArgs A) {
  __shared__ float4 sh_oth[kTJ];
  __shared__ int4 sh_vid[kTJ];
  __shared__ unsigned long long sh_end;
  const int64_t nB = A.nB;
  const int tid = threadIdx.x;
  for (int64_t i0 = (int64_t)blockIdx.x * kTI; i0 < nB; i0 += (int64_t)gridDim.x * kTI) {
    float ahi[2];
    float4 oi[2];
    int4 vi[2];
    int ki[2];
    // end of each box's sweep range relative to i0 (no box: empty range)
    int endl[2] = {tid + 1, kSweepThreads + tid + 1};
    int64_t end_max = i0;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
      const int64_t i = i0 + r * kSweepThreads + tid;
      ahi[r] = -__int_as_float(0x7F800000);   // no box: every test fails
      oi[r] = make_float4(0.f, 0.f, 0.f, 0.f);
      vi[r] = make_int4(-1, -1, -1, 0);
      if (i < nB) {
        ahi[r] = A.s_ahi[i];
        oi[r] = A.s_oth[i];
        vi[r] = A.s_vid[i];
        // first sorted index whose minimum exceeds ahi (binary search),
        // within the box's scene (batched scenes are contiguous runs)
        int64_t hi = nB;
        if (A.n_scenes > 0) {
          const int sid = A.bsid[vi[r].w];
          hi = A.voff[sid + 1] + A.eoff[sid + 1] + A.foff[sid + 1];
        }
        int64_t lo = i + 1;
        while (lo < hi) {
          const int64_t mid = (lo + hi) >> 1;
          if (A.s_alo[mid] <= ahi[r]) lo = mid + 1; else hi = mid;
        }
        endl[r] = (int)(lo - i0);
        end_max = lo > end_max ? lo : end_max;
      }
      ki[r] = box_kind(vi[r].w, A.nV, A.nE);
    }
    if (tid == 0) sh_end = (unsigned long long)i0;
    __syncthreads();
    atomicMax(&sh_end, (unsigned long long)end_max);
    __syncthreads();
    const int64_t jend = (int64_t)sh_end;
    const int li0 = tid, li1 = kSweepThreads + tid;   // local indices of the two boxes
    for (int64_t jt = i0 + 1; jt < jend; jt += kTJ) {
      __syncthreads();
      for (int k = tid; k < kTJ; k += kSweepThreads) {
        const int64_t j = jt + k;
        if (j < nB) {
          sh_oth[k] = A.s_oth[j];
          sh_vid[k] = A.s_vid[j];
        }
      }
      __syncthreads();
      const int cnt = (int)min((int64_t)kTJ, jend - jt);
      const int jl0 = (int)(jt - i0);      // local index of the tile's first box
      // box r tests j when li_r < jl < endl_r: in one sorted scene, j < end_r
      // is the same as min_a(j) <= max_a(i); unsigned form of the two tests
      const unsigned span0 = (unsigned)(endl[0] - li0 - 1), span1 = (unsigned)(endl[1] - li1 - 1);
      for (int k = 0; k < cnt; k += 4) {
        unsigned bits = 0;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const float4 oj = sh_oth[k + u];
          const int jl = jl0 + k + u;
          const bool h0 = ((unsigned)(jl - li0 - 1) < span0) & (oj.x <= oi[0].y) & (oi[0].x <= oj.y) &
                          (oj.z <= oi[0].w) & (oi[0].z <= oj.w);
          const bool h1 = ((unsigned)(jl - li1 - 1) < span1) & (oj.x <= oi[1].y) & (oi[1].x <= oj.y) &
                          (oj.z <= oi[1].w) & (oi[1].z <= oj.w);
          bits |= ((unsigned)h0 << (2 * u)) | ((unsigned)h1 << (2 * u + 1));
        }
        if (__any_sync(0xFFFFFFFFu, bits)) {
#pragma unroll
          for (int bb = 0; bb < 8; ++bb) {
            const bool hit = (bits >> bb) & 1u;
            if (__any_sync(0xFFFFFFFFu, hit)) {
              const int r = bb & 1;
              sweep_hit(A, hit, vi[r], ki[r], sh_vid[k + (bb >> 1)], nB);
            }
          }
        }
      }
    }
    __syncthreads();
  }
}

// Cell sweep (single-precision form), over the sorted box copies: a copy's
// sweep range ends at the first copy whose key exceeds (its cell, its maximum
// on the sweep axis), so it never leaves its cell, and a pair is kept only in
// the cell where, on each cell axis, one of its two copies lies in its box's
// first cell.  One thread per copy walks its own range (a few dozen copies):
// neighbouring lanes read neighbouring copies, so the loads coalesce and are
// served from L1, and a warp runs as many steps as its longest range.
// Pairs that pass the tests on the copies' extents, kinds and cells (hits,
// a few per lane and step, unevenly spread) queue in a per-warp shared list
// and are checked 32 at a time, one per lane, against the vertex-face /
// edge-edge rule and the shared-vertex filter.  Candidates collect in a
// per-warp shared buffer that is flushed with one atomic per 256 pairs; the
// exact FP64 test runs afterwards over the whole list (k_exact_filter).  The
// grid is persistent: the number of copies is known only on the device.
constexpr int kSupBuf = 256;

// End of a copy's sweep range: the first index after i whose sorted key
// exceeds the target.  The ranges are short, so the search gallops from i + 1
// (probes i+1, i+2, i+4, ...) and bisects only the last gap: a handful of
// neighbouring loads instead of a bisection over the whole array.
__device__ __forceinline__ int64_t range_end(const unsigned long long *__restrict__ key, int64_t i, int64_t n,
                                             unsigned long long target) {
  int64_t lo = i + 1, hi = i + 1, step = 1;   // keys in [i + 1, lo) are <= target
  while (hi < n && key[hi] <= target) {
    lo = hi + 1;
    hi += step;
    step <<= 1;
  }
  hi = hi < n ? hi : n;                        // key[hi] > target, or hi == n
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (key[mid] <= target) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// The same on (cell, ordered FP64 minimum) pairs, compared lexicographically.
__device__ __forceinline__ int64_t range_end64(const uint32_t *__restrict__ seg_of, const long long *__restrict__ key,
                                               int64_t i, int64_t n, uint32_t seg, long long target) {
  auto le = [&](int64_t j) {
    const uint32_t sj = seg_of[j];
    return sj < seg || (sj == seg && key[j] <= target);
  };
  int64_t lo = i + 1, hi = i + 1, step = 1;
  while (hi < n && le(hi)) {
    lo = hi + 1;
    hi += step;
    step <<= 1;
  }
  hi = hi < n ? hi : n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (le(mid)) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void sup_flush(const SweepArgs &A, uint2 *buf, int &cnt) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(&A.ctl->n_superset, (unsigned long long)cnt);
  base = __shfl_sync(0xFFFFFFFFu, base, 0);
  for (int k = lane; k < cnt; k += 32)
    if ((int64_t)(base + k) < A.sup_cap) A.sup[base + k] = buf[k];
  __syncwarp();
  cnt = 0;
}

// Candidates of a warp's pending hits, 32 at a time: lane k takes hit
// hb[k] (copy indices i, j) and runs the vertex-face / edge-edge rule and the
// shared-vertex filter on the two copies' boxes; survivors go to the warp's
// candidate buffer.
__device__ __forceinline__ void sweep_hits(const SweepArgs &A, const uint2 *hb, int nh, uint2 *buf, int &nbuf) {
  const int lane = threadIdx.x & 31;
  bool keep = false;
  uint2 pr = make_uint2(0u, 0u);
  if (lane < nh) {
    const uint2 h = hb[lane];
    int4 vi = A.s_vid[h.x], vj = A.s_vid[h.y];
    const unsigned fi = ((uint32_t)vi.w >> 30) & 3u, fj = ((uint32_t)vj.w >> 30) & 3u;
    vi.w &= 0x3FFFFFFF;
    vj.w &= 0x3FFFFFFF;
    bool vf;
    int p0, p1;
    if ((fi | fj) == 3u && candidate(vi, box_kind(vi.w, A.nV, A.nE), vj, A.nV, A.nE, vf, p0, p1)) {
      keep = true;
      pr = make_uint2((uint32_t)p0 | (vf ? 0x80000000u : 0u), (uint32_t)p1);
    }
  }
  const unsigned m = __ballot_sync(0xFFFFFFFFu, keep);
  if (m) {
    if (nbuf + __popc(m) > kSupBuf) sup_flush(A, buf, nbuf);
    if (keep) buf[nbuf + __popc(m & ((1u << lane) - 1u))] = pr;
    nbuf += __popc(m);
    __syncwarp();
  }
}

constexpr int kHitBuf = 160;   // a warp's pending hits: fewer than 32 + one step's at most 4 x 32

__global__ void __launch_bounds__(kSweepThreads) k_sweep_strips(SweepArgs A) {
  __shared__ uint2 sh_sup[kSweepThreads / 32][kSupBuf];
  __shared__ uint2 sh_hit[kSweepThreads / 32][kHitBuf];
  const int64_t n = (int64_t)*A.n_dev;
  const int lane = threadIdx.x & 31;
  uint2 *buf = sh_sup[threadIdx.x >> 5];
  uint2 *hb = sh_hit[threadIdx.x >> 5];
  int nbuf = 0;   // warp-uniform
  int nhit = 0;   // warp-uniform: pending hits in hb
  const int64_t ie = min(n, A.i_end);
  const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
  // a warp takes 32 consecutive copies per round (warp-uniform loop)
  for (int64_t base = A.i_begin + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < ie;
       base += wstride) {
    const int64_t i = base + lane;
    float4 oi = make_float4(0.f, 0.f, 0.f, 0.f);
    int4 vi = make_int4(-1, -1, -1, 0);
    unsigned fi = 0u;
    int64_t end = i + 1;   // no copy: empty range
    if (i < ie) {
      oi = A.s_oth[i];
      vi = A.s_vid[i];
      fi = ((uint32_t)vi.w >> 30) & 3u;   // first cell on each axis
      vi.w &= 0x3FFFFFFF;
      const unsigned long long target = (A.s_key[i] & 0xFFFFFFFF00000000ull) | f32_sort_key(A.s_ahi[i]);
      end = range_end(A.s_key, i, n, target);
    }
    const int ki = box_kind(vi.w, A.nV, A.nE);
    // the copy's range (i, end), 4 copies a step: neighbouring lanes read
    // neighbouring copies, so the loads coalesce and mostly hit L1; ids are
    // loaded only for pairs that pass the tests on extents, kinds and cells,
    // queued per warp and checked 32 at a time
    for (int64_t j0 = i + 1; __any_sync(0xFFFFFFFFu, j0 < end); j0 += 4) {
      unsigned hits = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (j0 + u < end) {
          // overlap on the two cell axes, a vertex-face or edge-edge pair
          // (kinds 0 + 2 or 1 + 1) and the one-cell reporting rule, before
          // the copy's ids are read
          const float4 oj = A.s_oth[j0 + u];
          const unsigned tj = A.s_tag[j0 + u];
          hits |= ((oj.x <= oi.y) & (oi.x <= oj.y) & (oj.z <= oi.w) & (oi.z <= oj.w) &
                   ((unsigned)ki + (tj & 3u) == 2u) & ((fi | (tj >> 2)) == 3u))
                      ? 1u << u
                      : 0u;
        }
      }
      // append this step's hits (copy i, copy j0 + u) to the warp's list
      const unsigned nh = (unsigned)__popc(hits);
      unsigned x = nh;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      const unsigned tot = __shfl_sync(0xFFFFFFFFu, x, 31);
      int pos = nhit + (int)(x - nh);
      while (hits) {
        const int u = __ffs((int)hits) - 1;
        hits &= hits - 1u;
        hb[pos++] = make_uint2((uint32_t)i, (uint32_t)(j0 + u));
      }
      nhit += (int)tot;
      __syncwarp();
      while (nhit >= 32) {
        nhit -= 32;
        sweep_hits(A, hb + nhit, 32, buf, nbuf);
        __syncwarp();
      }
    }
  }
  if (nhit) sweep_hits(A, hb, nhit, buf, nbuf);
  if (nbuf) sup_flush(A, buf, nbuf);
}

// FP64 cell sweep: k_sweep_strips on the FP64 extents (ordered int64 keys,
// exact comparisons).  A copy's range ends at the first copy with a larger
// (cell, minimum) than (its cell, its maximum).
__global__ void __launch_bounds__(kSweepThreads) k_sweep_strips64(SweepArgs A) {
  __shared__ uint2 sh_sup[kSweepThreads / 32][kSupBuf];
  __shared__ uint2 sh_hit[kSweepThreads / 32][kHitBuf];
  const int64_t n = (int64_t)*A.n_dev;
  const int lane = threadIdx.x & 31;
  uint2 *buf = sh_sup[threadIdx.x >> 5];
  uint2 *hb = sh_hit[threadIdx.x >> 5];
  int nbuf = 0;   // warp-uniform
  int nhit = 0;   // warp-uniform: pending hits in hb
  const int64_t ie = min(n, A.i_end);
  const int64_t wstride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = A.i_begin + (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < ie;
       base += wstride) {
    const int64_t i = base + lane;
    longlong2 o1 = make_longlong2(0, 0), o2 = make_longlong2(0, 0);
    int64_t end = i + 1;
    if (i < ie) {
      o1 = A.s_oth64c[2 * i];
      o2 = A.s_oth64c[2 * i + 1];
      end = range_end64(A.s_seg, A.s_key64, i, n, A.s_seg[i], A.s_ahi64c[i]);
    }
    for (int64_t j0 = i + 1; __any_sync(0xFFFFFFFFu, j0 < end); j0 += 4) {
      unsigned hits = 0;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (j0 + u < end) {
          const longlong2 p1 = A.s_oth64c[2 * (j0 + u)], p2 = A.s_oth64c[2 * (j0 + u) + 1];
          hits |= ((p1.x <= o1.y) & (o1.x <= p1.y) & (p2.x <= o2.y) & (o2.x <= p2.y)) ? 1u << u : 0u;
        }
      }
      // append this step's hits to the warp's list; check them 32 at a time
      const unsigned nh = (unsigned)__popc(hits);
      unsigned x = nh;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      const unsigned tot = __shfl_sync(0xFFFFFFFFu, x, 31);
      int pos = nhit + (int)(x - nh);
      while (hits) {
        const int u = __ffs((int)hits) - 1;
        hits &= hits - 1u;
        hb[pos++] = make_uint2((uint32_t)i, (uint32_t)(j0 + u));
      }
      nhit += (int)tot;
      __syncwarp();
      while (nhit >= 32) {
        nhit -= 32;
        sweep_hits(A, hb + nhit, 32, buf, nbuf);
        __syncwarp();
      }
    }
  }
  if (nhit) sweep_hits(A, hb, nhit, buf, nbuf);
  if (nbuf) sup_flush(A, buf, nbuf);
}

__global__ void k_reset_sweep(DevCtl *ctl) {
  ctl->n_vf = ctl->n_ee = ctl->n_superset = 0;
  ctl->sup_overflow = 0;
}

// Exact test of the strip sweep's candidates on the FP64 extents (ordered
// int64 keys), compacted into the vertex-face and edge-edge lists with one
// atomic per block and list.
constexpr int kFilterThreads = 256;
constexpr int kFilterItems = 8;

__global__ void __launch_bounds__(kFilterThreads) k_exact_filter(SweepArgs A) {
  __shared__ uint32_t wsum[2][kFilterThreads / 32];
  __shared__ unsigned long long sbase[2];
  const unsigned long long ns = A.ctl->n_superset;
  const int64_t n = (int64_t)min(ns, (unsigned long long)A.sup_cap);
  if (blockIdx.x == 0 && threadIdx.x == 0 && ns > (unsigned long long)A.sup_cap) {
    A.ctl->sup_overflow = 1;
    atomicCAS(&A.ctl->status, CCD_OK, CCD_ETRUNC);
  }
  const int64_t nB = A.nB;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  for (int64_t c0 = (int64_t)blockIdx.x * kFilterThreads * kFilterItems; c0 < n;
       c0 += (int64_t)gridDim.x * kFilterThreads * kFilterItems) {
    uint2 pr[kFilterItems];
    unsigned keep = 0, isvf = 0;
#pragma unroll
    for (int r = 0; r < kFilterItems; ++r) {
      const int64_t k = c0 + r * kFilterThreads + tid;
      pr[r] = make_uint2(0u, 0u);
      if (k < n) {
        pr[r] = A.sup[k];
        const bool vf = (pr[r].x >> 31) != 0;
        const int64_t a = pr[r].x & 0x7FFFFFFFu, b = pr[r].y;
        const int64_t bi = vf ? a : A.nV + a;
        const int64_t bj = vf ? A.nV + A.nE + b : A.nV + b;
        bool ov = true;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const long long ilo = A.lo64[x * nB + bi], ihi = A.hi64[x * nB + bi];
          const long long jlo = A.lo64[x * nB + bj], jhi = A.hi64[x * nB + bj];
          ov &= (jlo <= ihi) & (ilo <= jhi);
        }
        keep |= (unsigned)ov << r;
        isvf |= (unsigned)vf << r;
      }
    }
    // block-wide exclusive prefix of the kept vertex-face / edge-edge counts
    uint32_t cnt[2] = {(uint32_t)__popc(keep & isvf), (uint32_t)__popc(keep & ~isvf)};
    uint32_t incl[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      uint32_t x = cnt[t];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
      }
      incl[t] = x;
      if (lane == 31) wsum[t][w] = x;
    }
    __syncthreads();
    uint32_t before[2] = {0u, 0u};
    if (tid < 2) {
      uint32_t tot = 0;
      for (int k = 0; k < kFilterThreads / 32; ++k) tot += wsum[tid][k];
      sbase[tid] = tot ? atomicAdd(tid == 0 ? &A.ctl->n_vf : &A.ctl->n_ee, (unsigned long long)tot) : 0ull;
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < 2; ++t)
      for (int k = 0; k < w; ++k) before[t] += wsum[t][k];
    unsigned long long at[2] = {sbase[0] + before[0] + incl[0] - cnt[0], sbase[1] + before[1] + incl[1] - cnt[1]};
#pragma unroll
    for (int r = 0; r < kFilterItems; ++r) {
      if ((keep >> r) & 1u) {
        const int t = (isvf >> r) & 1u ? 0 : 1;
        int32_t *out = t == 0 ? A.vf_out : A.ee_out;
        const int64_t cap = t == 0 ? A.vf_cap : A.ee_cap;
        if ((int64_t)at[t] < cap) {
          const int64_t k = t == 1 && A.ee_rev ? cap - 1 - (int64_t)at[t] : (int64_t)at[t];
          out[2 * k] = (int32_t)(pr[r].x & 0x7FFFFFFFu);
          out[2 * k + 1] = (int32_t)pr[r].y;
        }
        ++at[t];
      }
    }
    __syncthreads();
  }
}

// Plain FP64 form: the sweep runs directly on the FP64 extents (ordered
// int64 keys, exact comparisons); no single-precision stage, no filter.
__global__ void __launch_bounds__(256) k_sweep64(SweepArgs A) {
  const int lane = threadIdx.x & 31;
  const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int64_t nB = A.nB;
  for (int64_t i = warp; i < nB; i += nwarps) {
    const long long ahi = A.s_ahi64[i];
    const longlong2 o1 = A.s_oth64[2 * i], o2 = A.s_oth64[2 * i + 1];
    const int4 vi = A.s_vid[i];
    const int ki = box_kind(vi.w, A.nV, A.nE);
    for (int64_t j0 = i + 1;; j0 += 32) {
      const int64_t j = j0 + lane;
      const bool in_a = j < nB && A.s_alo64[j] <= ahi;
      const unsigned run = __ballot_sync(0xFFFFFFFFu, in_a);
      bool is_vf = false, is_ee = false, sup = false;
      int p0 = 0, p1 = 0;
      if (in_a) {
        const longlong2 q1 = A.s_oth64[2 * j], q2 = A.s_oth64[2 * j + 1];
        if (q1.x <= o1.y && o1.x <= q1.y && q2.x <= o2.y && o2.x <= q2.y) {
          bool vf;
          if (candidate(vi, ki, A.s_vid[j], A.nV, A.nE, vf, p0, p1)) {
            sup = true;
            is_vf = vf;
            is_ee = !vf;
          }
        }
      }
      const unsigned bs = __ballot_sync(0xFFFFFFFFu, sup);
      if (bs && lane == 0) atomicAdd(&A.ctl->n_superset, (unsigned long long)__popc(bs));
      emit(A, is_vf, is_ee, p0, p1);
      if (run != 0xFFFFFFFFu) break;
    }
  }
}

}  // namespace ccd
