// Broad phase: boxes (Section "Construction of the Boxes") and
// sweep-and-prune (Section "Broad-Phase", Algorithm 2).
//
//   k_build_boxes   one thread per box: FP64 extents over t = 0 and t = 1 of
//                   the box's 1-3 vertices, single-precision box by directed
//                   rounding (round-down / round-up, the same float the paper's
//                   round-to-nearest-then-nextafterf rule gives), order-
//                   preserving integer keys of the FP64 extents for the exact
//                   test, and per-block sums for the centre variance.
//   k_axis_select   axis of largest centre variance (affects speed only).
//   k_radix_*       stable LSD radix sort of (key = ordered bits of the
//                   minimum on the sweep axis, value = box id), 4 x 8 bits.
//   k_gather_sorted box data in sorted order, structure of arrays.
//   k_sweep         one warp per sorted box i: lanes test i against
//                   j = i+1, i+2, ... while min_a(j) <= max_a(i), with the two
//                   other axes, the vertex-face / edge-edge rule, the
//                   shared-vertex filter and the exact FP64 box test fused;
//                   surviving pairs are appended with one atomic per warp.

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

namespace ccd {

__global__ void __launch_bounds__(kBuildThreads)
k_build_boxes(int64_t nV, int64_t nE, int64_t nF, const double *__restrict__ V0,
              const double *__restrict__ V1, const int32_t *__restrict__ E,
              const int32_t *__restrict__ F, BroadBufs B) {
  const int64_t nB = nV + nE + nF;
  const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  float c[3] = {0.f, 0.f, 0.f};
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
    }
    B.vid[b] = make_int4(ids[0], ids[1], ids[2], (int)b);
  }
  if (B.n_scenes > 0) {
    // batched scenes: the box's scene, and centre sums per scene (one atomic
    // per warp when the warp's boxes share a scene, which is the usual case)
    int sid = 0;
    if (b < nB)
      sid = b < nV ? scene_of(B.voff, B.n_scenes, b)
                   : (b < nV + nE ? scene_of(B.eoff, B.n_scenes, b - nV) : scene_of(B.foff, B.n_scenes, b - nV - nE));
    if (b < nB) B.bsid[b] = sid;
    const float v[6] = {c[0], c[1], c[2], c[0] * c[0], c[1] * c[1], c[2] * c[2]};
    const unsigned valid = __ballot_sync(0xFFFFFFFFu, b < nB);
    const unsigned peers = __match_any_sync(0xFFFFFFFFu, b < nB ? sid : -1);
    if (peers == 0xFFFFFFFFu && valid == 0xFFFFFFFFu) {
      float s6[6] = {v[0], v[1], v[2], v[3], v[4], v[5]};
#pragma unroll
      for (int i = 0; i < 6; ++i)
        for (int o = 16; o; o >>= 1) s6[i] += __shfl_xor_sync(0xFFFFFFFFu, s6[i], o);
      if ((threadIdx.x & 31) == 0)
        for (int i = 0; i < 6; ++i) atomicAdd(&B.ssum[i * B.n_scenes + sid], s6[i]);
    } else if (b < nB) {
      for (int i = 0; i < 6; ++i) atomicAdd(&B.ssum[i * B.n_scenes + sid], v[i]);
    }
    return;
  }
  // per-block sums of centres and squared centres (axis choice only)
  float s[6] = {c[0], c[1], c[2], c[0] * c[0], c[1] * c[1], c[2] * c[2]};
#pragma unroll
  for (int i = 0; i < 6; ++i)
    for (int o = 16; o; o >>= 1) s[i] += __shfl_xor_sync(0xFFFFFFFFu, s[i], o);
  __shared__ float red[kBuildThreads / 32][6];
  int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0)
    for (int i = 0; i < 6; ++i) red[w][i] = s[i];
  __syncthreads();
  if (threadIdx.x < 6) {
    float t = 0.f;
    for (int j = 0; j < kBuildThreads / 32; ++j) t += red[j][threadIdx.x];
    B.partials[6 * blockIdx.x + threadIdx.x] = t;
  }
}

__global__ void k_axis_select(const float *partials, int nblocks, int64_t nB, DevCtl *ctl) {
  __shared__ double acc[6][32];
  double s[6] = {0, 0, 0, 0, 0, 0};
  for (int i = threadIdx.x; i < nblocks; i += blockDim.x)
    for (int j = 0; j < 6; ++j) s[j] += (double)partials[6 * i + j];
  for (int j = 0; j < 6; ++j)
    for (int o = 16; o; o >>= 1) s[j] += __shfl_xor_sync(0xFFFFFFFFu, s[j], o);
  if ((threadIdx.x & 31) == 0)
    for (int j = 0; j < 6; ++j) acc[j][threadIdx.x >> 5] = s[j];
  __syncthreads();
  if (threadIdx.x == 0) {
    double t[6];
    for (int j = 0; j < 6; ++j) {
      t[j] = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t[j] += acc[j][w];
    }
    double inv = nB > 0 ? 1.0 / (double)nB : 0.0;
    int best = 0;
    double bv = -1.0;
    for (int a = 0; a < 3; ++a) {
      double mean = t[a] * inv;
      double var = t[3 + a] * inv - mean * mean;
      ctl->var_sum[a] = t[a];
      ctl->var_sum[3 + a] = t[3 + a];
      if (var > bv) { bv = var; best = a; }
    }
    ctl->axis = best;
  }
}

__global__ void k_make_keys(int64_t nB, const float *lo32, const DevCtl *ctl, uint32_t *keys, uint32_t *vals) {
  const int a = ctl->axis;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nB; i += (int64_t)gridDim.x * blockDim.x) {
    keys[i] = f32_sort_key(lo32[a * nB + i]);
    vals[i] = (uint32_t)i;
  }
}

// Batched scenes: axis of largest centre variance per scene.
__global__ void k_axis_select_scenes(BroadBufs B) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= B.n_scenes) return;
  const double n = (double)((B.voff[s + 1] - B.voff[s]) + (B.eoff[s + 1] - B.eoff[s]) + (B.foff[s + 1] - B.foff[s]));
  const double inv = n > 0 ? 1.0 / n : 0.0;
  int best = 0;
  double bv = -1.0;
  for (int a = 0; a < 3; ++a) {
    const double mean = (double)B.ssum[a * B.n_scenes + s] * inv;
    const double var = (double)B.ssum[(3 + a) * B.n_scenes + s] * inv - mean * mean;
    if (var > bv) { bv = var; best = a; }
  }
  B.saxis[s] = best;
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

// ---- radix sort: histogram / scan / stable scatter, 8 bits per pass --------

template <typename K>
__global__ void __launch_bounds__(kSortThreads)
k_radix_hist(const K *__restrict__ keys, int64_t n, int shift, uint32_t *hist, int ntiles) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    int64_t i = base + r * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];   // digit-major
}

// Row scan of the digit-major histogram: block d turns row d (the counts of
// digit d in every tile) into its exclusive prefix and stores the row total;
// the scatter adds the exclusive prefix of the totals (the digit's base).
__global__ void __launch_bounds__(256) k_radix_scan_rows(uint32_t *hist, int ntiles, uint32_t *totals) {
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t *row = hist + (int64_t)blockIdx.x * ntiles;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ntiles; base += 256) {
    const int i = base + tid;
    const uint32_t v = i < ntiles ? row[i] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wsum[warp] = x;
    __syncthreads();
    uint32_t before = carry;
    for (int w = 0; w < warp; ++w) before += wsum[w];
    const uint32_t excl = before + x - v;
    if (i < ntiles) row[i] = excl;
    __syncthreads();
    if (tid == 255) carry = excl + v;
    __syncthreads();
  }
  if (tid == 0) totals[blockIdx.x] = carry;
}

// Stable scatter of one tile: rounds of 256 consecutive keys; within a round
// each key's rank among equal digits comes from __match_any_sync (warp) plus
// the counts of earlier warps and earlier rounds.
template <typename K>
__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const K *__restrict__ keys_in, const uint32_t *__restrict__ vals_in, K *__restrict__ keys_out,
                uint32_t *__restrict__ vals_out, int64_t n, int shift, const uint32_t *__restrict__ offsets,
                int ntiles, const uint32_t *__restrict__ totals) {
  constexpr int kWarps = kSortThreads / 32;
  __shared__ uint32_t run[256];              // running position per digit
  __shared__ uint32_t wcnt[kWarps][256];     // per-warp digit counts of the round
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  {
    // digit base: exclusive scan of the 256 digit totals
    const uint32_t tot = totals[threadIdx.x];
    uint32_t x = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) wcnt[0][w] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int j = 0; j < w; ++j) before += wcnt[0][j];
    run[threadIdx.x] = before + x - tot + offsets[threadIdx.x * ntiles + blockIdx.x];
    __syncthreads();
  }
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int r = 0; r < kSortItems; ++r) {
    for (int j = 0; j < kWarps; ++j) wcnt[j][threadIdx.x] = 0;
    __syncthreads();
    int64_t i = base + r * kSortThreads + threadIdx.x;
    bool valid = i < n;
    K key = valid ? keys_in[i] : K(0);
    uint32_t val = valid ? vals_in[i] : 0;
    uint32_t d = valid ? (uint32_t)(key >> shift) & 0xFFu : 256u + lane;   // invalid lanes never match
    unsigned peers = __match_any_sync(0xFFFFFFFFu, d);
    uint32_t rank = __popc(peers & ((1u << lane) - 1u));
    if (valid && rank == 0) wcnt[w][d] = __popc(peers);
    __syncthreads();
    // exclusive prefix over warps for this thread's digit column
    uint32_t before = 0, tot = 0;
    {
      uint32_t col = threadIdx.x;
      uint32_t acc = 0;
      for (int j = 0; j < kWarps; ++j) {
        uint32_t c = wcnt[j][col];
        wcnt[j][col] = acc;
        acc += c;
      }
      tot = acc;
    }
    __syncthreads();
    if (valid) {
      before = wcnt[w][d];
      uint32_t pos = run[d] + before + rank;
      keys_out[pos] = key;
      vals_out[pos] = val;
    }
    __syncthreads();
    run[threadIdx.x] += tot;
    __syncthreads();
  }
}

template <typename K>
int radix_sort_t(K *keys[2], uint32_t *vals[2], int64_t n, uint32_t *hist, cudaStream_t s, int key_bits) {
  const int ntiles = (int)((n + kSortTile - 1) / kSortTile);
  uint32_t *totals = hist + 256 * (int64_t)ntiles;
  int cur = 0;
  const int bits = key_bits > 0 ? key_bits : (int)(8 * sizeof(K));
  for (int shift = 0; shift < bits; shift += 8) {
    k_radix_hist<K><<<ntiles, kSortThreads, 0, s>>>(keys[cur], n, shift, hist, ntiles);
    k_radix_scan_rows<<<256, 256, 0, s>>>(hist, ntiles, totals);
    k_radix_scatter<K><<<ntiles, kSortThreads, 0, s>>>(keys[cur], vals[cur], keys[cur ^ 1], vals[cur ^ 1], n, shift,
                                                       hist, ntiles, totals);
    cur ^= 1;
  }
  return cur;
}

int radix_sort(void *keys[2], uint32_t *vals[2], int key_bytes, int64_t n, uint32_t *hist, cudaStream_t s,
               int key_bits) {
  if (key_bytes == 4) {
    uint32_t *k[2] = {(uint32_t *)keys[0], (uint32_t *)keys[1]};
    return radix_sort_t<uint32_t>(k, vals, n, hist, s, key_bits);
  }
  unsigned long long *k[2] = {(unsigned long long *)keys[0], (unsigned long long *)keys[1]};
  return radix_sort_t<unsigned long long>(k, vals, n, hist, s, key_bits);
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
      A.ee_out[2 * at] = p0;
      A.ee_out[2 * at + 1] = p1;
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
