// Narrow phase: conservative interval bisection over (t, u, v) in FP64
// (Section "Narrow-Phase", Algorithm 3, ProcessInterval).
//
// GB300 design
//   * One persistent launch.  Every lane owns a unit of work (a whole query,
//     or a subtree of one) and walks it depth first, left half first.  The
//     split axis depends only on the interval's levels (see split_axis), so
//     every node at a given depth has the same levels and the DFS needs no
//     stack: the path is the binary expansion of the three numerators, kept
//     as bit masks of owed siblings and split axes for the 31 levels below
//     the depth at which the lane took its unit.
//   * Load balance at interval granularity: once every query has been
//     claimed, idle lanes take the shallowest owed sibling of a busy lane of
//     their warp, a warp hands its lanes' shallowest owed siblings to idle
//     warps of its block through a queue in shared memory, and every
//     32 x `budget` evaluations it hands them to a device-wide bounded MPMC
//     ring, which idle warps drain.  A near-degenerate query (tens of thousands of intervals)
//     is thus spread over many lanes, which is the point of the paper's
//     per-interval parallelism, without its level-synchronous launches.
//   * FP64 is the scarce unit on this GPU.  A full evaluation is 18 DFMA for
//     the two time ends (w, e1, e2 per axis), 24 DFMA for the corner hull and
//     3 DADD for the width test.  The hull needs only 2 of the 4 (u, v)
//     corners per time end and axis: rounding is monotone, so the minimum of
//     the computed corners is the corner picked by the signs of the computed
//     edge vectors, bit for bit the same as the minimum over all corners.
//     Almost every interval is decided without it, by the single-precision
//     filter, its certified ends and single FP64 corners (see inclusion32 and
//     the evaluation below).  Comparisons, min/max, interval ends and the
//     split rule run on the integer pipes.
//   * Earliest-TOI mode: one shared t* (ordered FP64 bits, atomicMin) prunes
//     every query; per-pair mode keeps t* per query.  Either way the result
//     for a query that hits no cap is independent of the traversal order: a
//     pruned interval starts at or after a t* that is already >= the final t*.
//
// Every wait is bounded; on expiry the kernel records CCD_ETIMEOUT and returns.
// Warps that find nothing to do for long enough leave, and the last one to
// leave records CCD_ETIMEOUT if any unit is still counted as unfinished.

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

namespace ccd {

namespace {

constexpr int kLevelCap = 53;
constexpr unsigned long long kInfBits = 0x7FF0000000000000ull;

struct QueryData {
  double c0[3][3];   // vector j at t = 0, axis x: VF w, e1, e2 / EE w, ea, eb
  double dc[3][3];   // value at t = 1 minus value at t = 0
  long long ebox_p[3], ebox_n[3];  // ordered keys of +ebox and -ebox
  unsigned long long K[3];         // split keys: bits of L_t, L_u, L_v (0: never)
  // single-precision filter (see inclusion32): rounded c0, dc and, per axis,
  // the decision thresholds tn, tm, wn and the bounds cc0, cdc of the
  // rounding of c0 and dc to float (summed over the three vectors)
  float c0f[3][3], dcf[3][3];
  float tn[3], tm[3], wn[3];
  float cc0[3], cdc[3];
};

__device__ __forceinline__ unsigned long long dbits(double d) {
  return (unsigned long long)__double_as_longlong(d);
}

// Conversions of doubles to float from their bits (integer operations only:
// on this GPU the conversion instructions share the narrow FP64 pipe).
// d2f_near: nearest, ties away from zero (error at most half an ulp); below
// the normal float range 0, from 2^128 up infinity.
__device__ __forceinline__ float d2f_near(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7FF) - 1023;
  if (E < -126) return __uint_as_float(sign);
  if (E > 127) return __uint_as_float(sign | 0x7F800000u);
  // round the 52-bit fraction to 23 bits; a carry out of the fraction raises
  // the exponent (to infinity from the top binade)
  const unsigned frac = (unsigned)(((b & 0x000FFFFFFFFFFFFFull) + (1ull << 28)) >> 29);
  return __uint_as_float(sign | (((unsigned)(E + 127) << 23) + frac));
}
// d2f_up / d2f_down for d >= 0: the float at or above / at or below d.
__device__ __forceinline__ float d2f_up(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  if (b == 0) return 0.f;
  const int E = (int)(b >> 52) - 1023;
  if (E < -126) return 0x1p-126f;
  if (E > 127) return __int_as_float(0x7F800000);
  const unsigned long long f = b & 0x000FFFFFFFFFFFFFull;
  const unsigned up = (f & ((1ull << 29) - 1)) != 0 ? 1u : 0u;
  return __uint_as_float(((unsigned)(E + 127) << 23) + (unsigned)(f >> 29) + up);
}
__device__ __forceinline__ float d2f_down(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d);
  const int E = (int)(b >> 52) - 1023;
  if (E < -126) return 0.f;
  if (E > 127) return __int_as_float(0x7F7FFFFF);
  return __uint_as_float(((unsigned)(E + 127) << 23) + (unsigned)((b & 0x000FFFFFFFFFFFFFull) >> 29));
}

// An upper bound of |d2f_near(d) - d|: 0 when d is a float (its low 29
// significand bits are zero and it lies in the normal float range), else one
// float ulp at d's exponent; 2^-126 below the normal range (d2f_near gives 0
// there), infinity from 2^127 up.  Integer operations only.
__device__ __forceinline__ float to_float_error(double d) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(d) & 0x7FFFFFFFFFFFFFFFull;
  if (b == 0) return 0.f;
  const int E = (int)(b >> 52) - 1023;
  if (E > 126) return __int_as_float(0x7F800000);   // may round to infinity
  if (E < -126) return 0x1p-126f;
  if ((b & ((1ull << 29) - 1)) == 0) return 0.f;
  const int fe = E - 23;   // float ulp at exponent E
  return fe >= -126 ? __int_as_float((fe + 127) << 23) : __int_as_float(1 << (fe + 149));
}

// The error-box term of one coordinate pair: bits of max(|x0|, |x1|) (the
// magnitudes of finite doubles order like their bits).
__device__ __forceinline__ unsigned long long abs_max_bits(double a, double b) {
  const unsigned long long x = dbits(a) & 0x7FFFFFFFFFFFFFFFull, y = dbits(b) & 0x7FFFFFFFFFFFFFFFull;
  return x > y ? x : y;
}
constexpr unsigned long long kM0 = 0x03F0000000000000ull;   // 2^-960, floor of the coordinate bound m
// eps = m * 48 * 2^-53 from the bits of m
__device__ __forceinline__ double eps_of(unsigned long long m) {
  return __dmul_rn(__longlong_as_double((long long)m), 0x1.8p-48);
}

// One axis of the second half of the per-query set-up, from the three
// vectors' c0, dc on that axis and the error term eps = 48 * 2^-53 m: the
// error box e = eps + min_sep moved one ulp up, the axis's part of the time
// weight L_t (bits of sum_j |dc_j|) and the single-precision filter data.
// Rounding of eps + min_sep is monotone, so the box of a query is the
// largest box of its primitives when eps comes as the largest of theirs.
struct AxisSetup {
  double e;                      // error box half-width on the axis
  float c0f[3], dcf[3];          // c0, dc rounded to float
  float tn, tm, wn, cc0, cdc;    // filter thresholds and rounding bounds
  unsigned long long st;         // bits of |dc_0| + |dc_1| + |dc_2|
};

__device__ __forceinline__ void setup_axis(AxisSetup &o, const double c0[3], const double dc[3], double eps,
                                           double min_sep, bool no_sep, double delta) {
  double e = no_sep ? eps : __dadd_rn(eps, min_sep);   // (no_sep: min_sep == 0, and eps + 0 is eps)
  e = __longlong_as_double(__double_as_longlong(e) + 1);       // one ulp up
  o.e = e;
  // FP32 filter bounds (derivations at inclusion32).  With S the sum over
  // the three vectors of |c0| + |dc| on this axis, the FP32 and FP64 hulls
  // are less than e32 = 8 * 2^-24 * max(S, 2^-100) apart, and the FP64 hull
  // is within e64 = 4 * 2^-53 S (+ 2^-1060 for subnormals) of R, the hull
  // evaluated exactly from c0 and dc.  A decision taken on the FP32 hull must
  // hold for the FP64 hull:
  //   tm = e + eps + e32  (beyond it, the FP64 hull misses or sticks out of C;
  //                        eps is spare margin)
  //   wn = (delta (1 + 2^-50) + 2 eps + 2 e32)(1 + 2^-23)  (an FP32 width at or
  //        above it means an FP64 width at or above delta)
  //   tn = e - e64, rounded down  (an upper bound of R's low end at or below
  //        it means the FP64 low end is at most e: no miss on that side)
  // (all in single precision, every operation rounded toward the safe side,
  // so each threshold is at least (tn: at most) its exact value; S from
  // |c0| <= |float(c0)| + cc0-term; delta (1 + 2^-50) is bounded by
  // delta (1 + 2^-23); 2^-149 stands in for 2^-1060)
  float s32 = 0.f, cc0 = 0.f, cdc = 0.f;
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const float cf = d2f_near(c0[j]), df = d2f_near(dc[j]);
    const float ec = to_float_error(c0[j]), ed = to_float_error(dc[j]);
    o.c0f[j] = cf;
    o.dcf[j] = df;
    cc0 = __fadd_ru(cc0, ec);
    cdc = __fadd_ru(cdc, ed);
    s32 = __fadd_ru(s32, __fadd_ru(fabsf(cf), ec));
    s32 = __fadd_ru(s32, __fadd_ru(fabsf(df), ed));
  }
  o.cc0 = cc0;
  o.cdc = cdc;
  s32 = fmaxf(s32, 0x1p-100f);
  const float e32 = __fmul_ru(s32, 8.0f * 0x1p-24f);
  const float eps32 = d2f_up(eps), e_32 = d2f_up(e);
  const float e64 = __fmaf_ru(s32, 0x1p-51f, 0x1p-149f);
  o.tn = __fsub_rd(d2f_down(e), e64);
  o.tm = __fadd_ru(__fadd_ru(e_32, eps32), e32);
  const float d32 = __fmul_ru(d2f_up(delta), 1.0f + 0x1p-23f);
  const float wn = __fadd_ru(__fadd_ru(d32, __fmul_ru(2.0f, eps32)), __fmul_ru(2.0f, e32));
  o.wn = __fmul_ru(wn, 1.0f + 0x1p-23f);
  double st = __dadd_rn(dabs_int(dc[0]), dabs_int(dc[1]));
  st = __dadd_rn(st, dabs_int(dc[2]));
  o.st = dbits(st);
}

constexpr unsigned long long kKeyFloor = 0x0DF0000000000000ull;   // 2^-800: smaller split weights never split

// Second half of the per-query set-up, from c0, dc (already in Q), eps per
// axis and the split weights L_u, L_v (bits): setup_axis on each axis, the
// time weight L_t and the split keys.
__device__ void setup_tail(QueryData &Q, const double eps_x[3], unsigned long long Lu, unsigned long long Lv,
                           double min_sep, double delta) {
  unsigned long long Lt = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double c0[3] = {Q.c0[0][x], Q.c0[1][x], Q.c0[2][x]}, dc[3] = {Q.dc[0][x], Q.dc[1][x], Q.dc[2][x]};
    AxisSetup o;
    setup_axis(o, c0, dc, eps_x[x], min_sep, min_sep == 0.0, delta);
    Q.ebox_p[x] = f64_ord(o.e);
    Q.ebox_n[x] = f64_ord(-o.e);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      Q.c0f[j][x] = o.c0f[j];
      Q.dcf[j][x] = o.dcf[j];
    }
    Q.cc0[x] = o.cc0;
    Q.cdc[x] = o.cdc;
    Q.tn[x] = o.tn;
    Q.tm[x] = o.tm;
    Q.wn[x] = o.wn;
    Lt = o.st > Lt ? o.st : Lt;
  }
  Q.K[0] = Lt < kKeyFloor ? 0 : Lt;
  Q.K[1] = Lu < kKeyFloor ? 0 : Lu;
  Q.K[2] = Lv < kKeyFloor ? 0 : Lv;
}

// Bits of max over axes and t in {0, 1} of |c0 + t dc| for one vector (the
// value at t = 1 as c0 + dc, rounded): the split weight L_u or L_v.
__device__ __forceinline__ unsigned long long edge_weight(const double c0[3], const double dc[3]) {
  unsigned long long L = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const unsigned long long a = abs_max_bits(c0[x], __dadd_rn(c0[x], dc[x]));
    L = a > L ? a : L;
  }
  return L;
}

// Per-query set-up; the reading of the error box and split weights matches the
// oracle's setup_query.  ids: VF (P, T0, T1, T2), EE (A0, A1, B0, B1).
__device__ void setup_query(QueryData &Q, bool vf, const int ids[4], const double *__restrict__ V0,
                            const double *__restrict__ V1, int64_t nV, double min_sep, double delta) {
  double x0[4][3], x1[4][3];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      x0[k][x] = __ldg(&V0[x * nV + ids[k]]);
      x1[k][x] = __ldg(&V1[x * nV + ids[k]]);
    }
  // vector j = X - Y: VF (P - T0, T1 - T0, T2 - T0); EE (A0 - B0, A1 - A0, B1 - B0)
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const double X0[3] = {x0[0][x], vf ? x0[2][x] : x0[1][x], x0[3][x]};
    const double Y0[3] = {vf ? x0[1][x] : x0[2][x], vf ? x0[1][x] : x0[0][x], vf ? x0[1][x] : x0[2][x]};
    const double X1[3] = {x1[0][x], vf ? x1[2][x] : x1[1][x], x1[3][x]};
    const double Y1[3] = {vf ? x1[1][x] : x1[2][x], vf ? x1[1][x] : x1[0][x], vf ? x1[1][x] : x1[2][x]};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      double a = __dsub_rn(X0[j], Y0[j]);
      double b = __dsub_rn(X1[j], Y1[j]);
      Q.c0[j][x] = a;
      Q.dc[j][x] = __dsub_rn(b, a);
    }
  }
  double eps[3];
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    unsigned long long m = kM0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned long long a = abs_max_bits(x0[k][x], x1[k][x]);
      m = a > m ? a : m;
    }
    eps[x] = eps_of(m);
  }
  setup_tail(Q, eps, edge_weight(Q.c0[1], Q.dc[1]), edge_weight(Q.c0[2], Q.dc[2]), min_sep, delta);
}

// Per-primitive set-up (the parts of a query's set-up that depend on one
// primitive only, computed once per primitive instead of once per query):
//   vertex v:  eps[3] of its coordinates, padded to 4 words;
//   edge e:    c0[3], dc[3] of A1 - A0, eps[3] over its two vertices, the
//              split weight of the vector (kEdgeWords words);
//   face f:    c0[3], dc[3] of T1 - T0 and of T2 - T0, eps[3] over its three
//              vertices, the two split weights, padded (kFaceWords words).
// The same FP64 operations on the same operands as setup_query, so every
// value is bit-identical; eps of a query is the largest of its primitives'
// (rounding of m * 48 * 2^-53 is monotone in m).
constexpr int kVertWords = 4, kEdgeWords = 10, kFaceWords = 18;

__device__ __forceinline__ void load_pos(const double *__restrict__ V0, const double *__restrict__ V1, int64_t nV,
                                         int id, double p0[3], double p1[3]) {
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    p0[x] = __ldg(&V0[x * nV + id]);
    p1[x] = __ldg(&V1[x * nV + id]);
  }
}

// vector Y -> X: c0 = X0 - Y0, dc = (X1 - Y1) - c0
__device__ __forceinline__ void vec_of(const double X0[3], const double X1[3], const double Y0[3], const double Y1[3],
                                       double c0[3], double dc[3]) {
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    c0[x] = __dsub_rn(X0[x], Y0[x]);
    dc[x] = __dsub_rn(__dsub_rn(X1[x], Y1[x]), c0[x]);
  }
}

__device__ __forceinline__ void store2(double *p, double a, double b) { *(double2 *)p = make_double2(a, b); }

__device__ __forceinline__ double dmax_pos(double a, double b) {   // both > 0
  return dbits(a) > dbits(b) ? a : b;
}

// Split rule (reading): axis with the largest L_k * 2^-l_k, ties t, u, v;
// axes at the level cap or with L_k = 0 are never split.  L_k >= 2^-800 and
// l_k <= 53, so bits(L_k) - (l_k << 52) are the bits of L_k * 2^-l_k.
//
// last_axis: the axis split last on the way to a node with these levels.  The
// splits taken so far are the largest values L_k 2^-j (j < l_k) in the order
// (value descending, axis ascending), so the last one is the smallest of
// L_k 2^-(l_k - 1), ties to the highest axis.

// An interval [n_k / 2^l_k, (n_k + 1) / 2^l_k] on t (k = 0), u (1), v (2),
// kept in scalar fields so that a runtime axis never indexes an array.
struct Node {
  uint64_t n0, n1, n2;
  int l0, l1, l2;
  __device__ __forceinline__ uint64_t n(int a) const { return a == 0 ? n0 : (a == 1 ? n1 : n2); }
  __device__ __forceinline__ void down_left(int a) {   // to the left child along a
    if (a == 0) { n0 <<= 1; ++l0; } else if (a == 1) { n1 <<= 1; ++l1; } else { n2 <<= 1; ++l2; }
  }
  __device__ __forceinline__ void up(int a) {          // to the parent along a
    if (a == 0) { n0 >>= 1; --l0; } else if (a == 1) { n1 >>= 1; --l1; } else { n2 >>= 1; --l2; }
  }
  __device__ __forceinline__ void add(int a, uint64_t v) {
    if (a == 0) n0 += v; else if (a == 1) n1 += v; else n2 += v;
  }
  __device__ __forceinline__ int depth() const { return l0 + l1 + l2; }
};

// Interval ends as integers: n / 2^l scaled by 2^53 (exact, below 2^53 for
// n < 2^l, l <= 53), and a t* given by its bits as ceil(t* 2^53), at most
// 2^53.  Then t_lo >= t* is s53(n, l) >= ceil53(t*), and the vertex-face
// simplex test u_lo + v_lo > 1 is s53(n1, l1) + s53(n2, l2) > 2^53.
__device__ __forceinline__ uint64_t s53(uint64_t n, int l) { return n << (53 - l); }
__device__ __forceinline__ uint64_t ceil53(unsigned long long cb) {
  if (cb >= 0x3FF0000000000000ull) return 1ull << 53;   // t* >= 1 (or +inf): nothing starts there
  if (cb == 0) return 0;
  const int sh = 1022 - (int)(cb >> 52);                // t* = m 2^(E - 52), times 2^53 = m >> sh
  const uint64_t m = (cb & 0x000FFFFFFFFFFFFFull) | ((cb >> 52) ? (1ull << 52) : 0ull);
  if (sh >= 64) return 1;                               // 0 < t* < 2^-53
  const uint64_t q = m >> sh;
  return (q << sh) == m ? q : q + 1;
}
__device__ __forceinline__ bool outside_simplex(const Node &N) {
  return s53(N.n1, N.l1) + s53(N.n2, N.l2) > (1ull << 53);
}

__device__ __forceinline__ int split_axis(const unsigned long long K[3], const Node &N) {
  const int l[3] = {N.l0, N.l1, N.l2};
  int best = -1;
  unsigned long long bv = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (K[k] == 0 || l[k] >= kLevelCap) continue;
    unsigned long long v = K[k] - ((unsigned long long)l[k] << 52);
    if (best < 0 || v > bv) { best = k; bv = v; }
  }
  return best;
}

__device__ __forceinline__ int last_axis(const unsigned long long K[3], const Node &N) {
  const int l[3] = {N.l0, N.l1, N.l2};
  int best = -1;
  unsigned long long bv = 0;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    if (l[k] == 0) continue;
    unsigned long long v = K[k] - ((unsigned long long)(l[k] - 1) << 52);
    if (best < 0 || v <= bv) { best = k; bv = v; }
  }
  return best;
}

// The shallowest pending right sibling on the path from the unit's root to
// node N (depth `depth`) that starts before `cut` (bits of the current t*):
// the largest subtree the lane still owes.  Returns its depth (0 if none) and
// the sibling in S.  Pending siblings above it start at or after t*, so they
// would be pruned: a lane that hands S off and keeps only what lies below
// S's depth loses nothing (their accepts could not lower t*).
__device__ __forceinline__ int shallowest_pending(const unsigned long long K[3], const Node &N, int depth,
                                                  int root_depth, unsigned long long cut, Node &S) {
  Node W = N;
  int found = 0;
  const uint64_t cut53 = ceil53(cut);
  for (int d = depth; d > root_depth; --d) {
    int a = last_axis(K, W);
    if ((W.n(a) & 1) == 0) {
      const uint64_t n0 = a == 0 ? W.n0 + 1 : W.n0;   // the sibling's t numerator
      if (s53(n0, W.l0) < cut53) {
        S = W;
        S.add(a, 1);
        found = d;
      }
    }
    W.up(a);
  }
  return found;
}

// shallowest_pending on the path masks of the narrow kernel (units no more
// than 31 levels below the masks' base depth; depth, root_depth and the
// returned depth count from that base): pend bit d marks an owed right
// sibling at depth d, (axhi, axlo) bit d the axis split to reach depth d.
// The owed siblings are visited from the shallowest; the first that starts
// before `cut` is returned.
__device__ __forceinline__ int shallowest_owed(const Node &N, int depth, int root_depth, unsigned pend,
                                               unsigned axlo, unsigned axhi, unsigned long long cut, Node &S) {
  const uint64_t cut53 = ceil53(cut);
  unsigned m = pend & (root_depth >= 31 ? 0u : ~0u << (root_depth + 1));
  const unsigned upto = depth >= 31 ? ~0u : (2u << depth) - 1u;
  while (m) {
    const int d = __ffs((int)m) - 1;
    const unsigned r = upto & (d >= 31 ? 0u : ~0u << (d + 1));
    const int c1 = __popc(r & axlo & ~axhi), c2 = __popc(r & axhi);
    const int c0 = depth - d - c1 - c2;
    Node W{N.n0 >> c0, N.n1 >> c1, N.n2 >> c2, N.l0 - c0, N.l1 - c1, N.l2 - c2};
    const int a = (int)((axlo >> d) & 1u) | ((int)((axhi >> d) & 1u) << 1);
    if (s53(a == 0 ? W.n0 + 1 : W.n0, W.l0) < cut53) {
      S = W;
      S.add(a, 1);
      return d;
    }
    m &= m - 1u;
  }
  return 0;
}

struct Box3 {
  double lo[3], hi[3];
};

// B_F(I): the hull of F at the corners of I, from 2 corners per time end.
__device__ __forceinline__ void inclusion(const QueryData &Q, bool vf, double tl, double tr, double ul,
                                          double ur, double vl, double vr, Box3 &B) {
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    double lo = 0.0, hi = 0.0;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      double tt = it ? tr : tl;
      double w = fma(tt, Q.dc[0][x], Q.c0[0][x]);
      double a = fma(tt, Q.dc[1][x], Q.c0[1][x]);
      double b = fma(tt, Q.dc[2][x], Q.c0[2][x]);
      double fmin, fmax;
      bool ap = __double_as_longlong(a) > 0;  // a > +0 (a is never NaN)
      bool bp = __double_as_longlong(b) > 0;
      if (vf) {
        // f = (w - v e2) - u e1: inner v term, outer u term
        double gmin = fma(-(bp ? vr : vl), b, w);
        double gmax = fma(-(bp ? vl : vr), b, w);
        fmin = fma(-(ap ? ur : ul), a, gmin);
        fmax = fma(-(ap ? ul : ur), a, gmax);
      } else {
        // f = (w + u ea) - v eb: inner u term, outer v term
        double gmin = fma(ap ? ul : ur, a, w);
        double gmax = fma(ap ? ur : ul, a, w);
        fmin = fma(-(bp ? vr : vl), b, gmin);
        fmax = fma(-(bp ? vl : vr), b, gmax);
      }
      if (it == 0) {
        lo = fmin;
        hi = fmax;
      } else {
        lo = dmin_int(lo, fmin);
        hi = dmax_int(hi, fmax);
      }
    }
    B.lo[x] = lo;
    B.hi[x] = hi;
  }
}

// Single-precision hull of F over an interval with every level <= 24 (its
// ends are then exact floats), same expression tree and corner selection as
// inclusion().  Error bound on one axis, with u = 2^-24, c0 and dc the FP64
// set-up values, S_j = |c0_j| + |dc_j| for the vectors j = w, e1, e2 and
// S = S_w + S_1 + S_2 (t, u, v in [0, 1]; second-order terms dropped):
//   c_j(t) = fma(t, dcf, c0f) with c0f, dcf rounded from c0, dc:
//       |c_j(t) - (c0 + t dc)| <= u |dc| + u |c0| + u S_j = 2 u S_j;
//   inner term g = fma(-v, c_k, w), one rounding of a value below S_w + S_k:
//       2 u S_w + 2 u S_k + u (S_w + S_k) = 3 u (S_w + S_k);
//   corner f = fma(-u, c_i, g): 3 u (S_w + S_k) + 2 u S_i + u S <= 4 u S;
//   corner choice: a sign of c_i(t) taken wrong in FP32 means |c_i| <= 2 u S_i,
//       and the chosen corner is then within 2 u S_i of the extreme one, so
//       both choices together add at most 2 u (S_1 + S_2).
// That is at most 6 u S from R, the hull evaluated exactly from the FP64 c0
// and dc.  The same steps in FP64 (no conversion, unit 2^-53) put inclusion()
// within 4 * 2^-53 S of R.  So on every axis the FP32 and FP64 hulls are less
// than e32 = 8 u S apart, whatever the size of the coordinates: S is built
// from differences of vertex positions, not from the positions.
//
// e32 is too wide to settle a hull end that lies at or near 0, and such ends
// are common: start positions in a common plane give corners that are exactly
// 0 at t = 0, and a vertex on a grid line of the other element gives corners
// where nonzero terms cancel exactly.  For those the kernel also evaluates the
// selected low and high corners in interval arithmetic: c_j(t) from
// fma_rd / fma_ru of (t, dcf, c0f), the corner from outward-rounded fmas of
// those ends, then widened by conv(t) = cc0 + t cdc, with cc0, cdc bounding
// the rounding of c0 and dc to float summed over the vectors (the corner's
// multipliers are at most 1).  L = min over t of the upper bound of R at the
// low corner bounds R's low end from above (R's low end is at most R at any
// corner); H likewise from below.  Where every operation is exact the two
// directions agree and the bound is the exact value, 0 at such an end.  The
// FP64 low end is then at most L + e64, and the kernel compares L against
// tn = e - e64.
struct Box3f {
  float lo[3], hi[3];   // the FP32 hull
  float L[3], H[3];     // upper bound of R's low end, lower bound of its high end
  unsigned tb;          // t end of the FP64 corner check, bit x for a low end, bit 3 + x for a
                        // high end (1: right end).  Left end throughout: taking the end the
                        // certified bound came from settled no more ends on the cloth and cost
                        // more.
};

__device__ __forceinline__ void inclusion32(const float c0f[3][3], const float dcf[3][3], const float cc0[3],
                                            const float cdc[3], bool vf, float tl, float tr, float ul, float ur,
                                            float vl, float vr, Box3f &B) {
  B.tb = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    float lo = 0.f, hi = 0.f, L = 0.f, H = 0.f;
#pragma unroll
    for (int it = 0; it < 2; ++it) {
      const float tt = it ? tr : tl;
      const float w = fmaf(tt, dcf[0][x], c0f[0][x]);
      const float a = fmaf(tt, dcf[1][x], c0f[1][x]);
      const float b = fmaf(tt, dcf[2][x], c0f[2][x]);
      const bool ap = a > 0.f, bp = b > 0.f;
      // multipliers of the low and high corners: u on a, v on b
      float ulo, uhi, vlo, vhi;
      float fmin, fmax;
      if (vf) {
        vlo = bp ? vr : vl;
        vhi = bp ? vl : vr;
        ulo = ap ? ur : ul;
        uhi = ap ? ul : ur;
        fmin = fmaf(-ulo, a, fmaf(-vlo, b, w));
        fmax = fmaf(-uhi, a, fmaf(-vhi, b, w));
      } else {
        ulo = ap ? ul : ur;
        uhi = ap ? ur : ul;
        vlo = bp ? vr : vl;
        vhi = bp ? vl : vr;
        fmin = fmaf(-vlo, b, fmaf(ulo, a, w));
        fmax = fmaf(-vhi, b, fmaf(uhi, a, w));
      }
      // certified ends: the same corners in interval arithmetic, every
      // operation rounded outward, widened by the rounding of c0, dc to float
      const float wu = __fmaf_ru(tt, dcf[0][x], c0f[0][x]), wd = __fmaf_rd(tt, dcf[0][x], c0f[0][x]);
      const float au = __fmaf_ru(tt, dcf[1][x], c0f[1][x]), ad = __fmaf_rd(tt, dcf[1][x], c0f[1][x]);
      const float bu = __fmaf_ru(tt, dcf[2][x], c0f[2][x]), bd = __fmaf_rd(tt, dcf[2][x], c0f[2][x]);
      const float conv = __fmaf_ru(tt, cdc[x], cc0[x]);
      float Lt, Ht;
      if (vf) {
        Lt = __fmaf_ru(-ulo, ad, __fmaf_ru(-vlo, bd, wu));
        Ht = __fmaf_rd(-uhi, au, __fmaf_rd(-vhi, bu, wd));
      } else {
        Lt = __fmaf_ru(-vlo, bd, __fmaf_ru(ulo, au, wu));
        Ht = __fmaf_rd(-vhi, bu, __fmaf_rd(uhi, ad, wd));
      }
      Lt = __fadd_ru(Lt, conv);
      Ht = __fsub_rd(Ht, conv);
      lo = it ? fminf(lo, fmin) : fmin;
      hi = it ? fmaxf(hi, fmax) : fmax;
      L = it ? fminf(L, Lt) : Lt;
      H = it ? fmaxf(H, Ht) : Ht;
    }
    B.lo[x] = lo;
    B.hi[x] = hi;
    B.L[x] = L;
    B.H[x] = H;
  }
}

// A non-negative float that is 0 or normal, as a double (exact), from bits.
__device__ __forceinline__ double f2d_exact(float f) {
  const unsigned b = __float_as_uint(f);
  if (b == 0) return 0.0;
  const unsigned long long e = (unsigned long long)(b >> 23) + (1023 - 127);
  return __longlong_as_double((long long)((e << 52) | ((unsigned long long)(b & 0x7FFFFFu) << 29)));
}

// n / 2^l as a float, exact for n <= 2^24 and l <= 24, assembled from bits.
__device__ __forceinline__ float dyadic32(uint64_t n, int l) {
  // n <= 2^24 converts exactly; scaling by 2^-l moves the exponent only
  const float f = __uint2float_rn((unsigned)n);
  return n == 0 ? 0.f : __int_as_float(__float_as_int(f) - (l << 23));
}

// The FP64 part of a lane's query, kept in shared memory (structure of
// arrays: consecutive lanes hit consecutive banks).
struct SharedQuery {
  double c0[9][kNarrowThreads];
  double dc[9][kNarrowThreads];
  long long ep[3][kNarrowThreads], en[3][kNarrowThreads];
  float cc0[3][kNarrowThreads], cdc[3][kNarrowThreads];   // used by the FP32 filter
};

__device__ __forceinline__ void put_shared(SharedQuery &S, int tid, const QueryData &Q) {
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      S.c0[3 * j + x][tid] = Q.c0[j][x];
      S.dc[3 * j + x][tid] = Q.dc[j][x];
    }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    S.ep[x][tid] = Q.ebox_p[x];
    S.en[x][tid] = Q.ebox_n[x];
    S.cc0[x][tid] = Q.cc0[x];
    S.cdc[x][tid] = Q.cdc[x];
  }
}

__device__ __forceinline__ void copy_shared(SharedQuery &S, int dst, int src) {
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    S.c0[k][dst] = S.c0[k][src];
    S.dc[k][dst] = S.dc[k][src];
  }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    S.ep[x][dst] = S.ep[x][src];
    S.en[x][dst] = S.en[x][src];
    S.cc0[x][dst] = S.cc0[x][src];
    S.cdc[x][dst] = S.cdc[x][src];
  }
}

__device__ __forceinline__ void inclusion_shared(const SharedQuery &S, int tid, bool vf, double tl, double tr,
                                                 double ul, double ur, double vl, double vr, Box3 &B) {
  QueryData Q;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Q.c0[j][x] = S.c0[3 * j + x][tid];
      Q.dc[j][x] = S.dc[3 * j + x][tid];
    }
  inclusion(Q, vf, tl, tr, ul, ur, vl, vr, B);
}

// ---- bounded MPMC ring of exported intervals -------------------------------
// Cell: sequence number + interval.  A cell at position p holds data when
// seq == p + 1 and is free for position p + cap once its reader stores
// seq = p + cap.  Writers first reserve all the positions they need with one
// CAS on `tail`, and only while every reserved position is below
// head + cap: each such position's previous occupant has already been popped,
// so a writer never waits on a reader that has not started.  A hand-off that
// does not fit is not made (the lane keeps the work), so pushes cannot block.

__device__ __forceinline__ unsigned long long pack1(uint64_t n, int l) {
  return n | ((unsigned long long)l << 54);
}

// Reserve m consecutive positions if the ring then stays below `limit`
// occupied slots; returns the first position or ~0ull.
__device__ unsigned long long ring_reserve(unsigned long long *tail, const unsigned long long *head,
                                           unsigned long long m, unsigned long long limit) {
  for (int tries = 0; tries < 32; ++tries) {
    unsigned long long t = ld_relaxed_u64(tail);
    unsigned long long h = ld_relaxed_u64(head);
    if (t - h + m > limit) return ~0ull;
    if (atomicCAS(tail, t, t + m) == t) return t;
  }
  return ~0ull;
}

// Write one interval at a reserved position.  The wait is for a reader that
// has already popped the previous occupant and is copying it out.
__device__ bool ring_write(RingCell *ring, unsigned long long mask, unsigned long long pos, uint32_t q,
                           const Node &N, int *status) {
  RingCell *c = &ring[pos & mask];
  for (int spin = 0; ld_acquire_u64(&c->seq) != pos; ++spin) {
    if (spin > (1 << 22)) {
      atomicExch(status, CCD_ETIMEOUT);
      return false;
    }
    __nanosleep(32);
  }
  c->w[0] = pack1(N.n0, N.l0);
  c->w[1] = pack1(N.n1, N.l1);
  c->w[2] = pack1(N.n2, N.l2);
  c->q = q;
  st_release_u64(&c->seq, pos + 1);
  return true;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void query_ids(int64_t q, int64_t n_vf, const int32_t *__restrict__ vfp,
                                          const int32_t *__restrict__ eep, const int32_t *__restrict__ E,
                                          const int32_t *__restrict__ F, int ids[4], bool &vf) {
  if (q < n_vf) {
    vf = true;
    int v = __ldg(&vfp[2 * q]);
    int f = __ldg(&vfp[2 * q + 1]);
    ids[0] = v;
    ids[1] = __ldg(&F[3 * f]);
    ids[2] = __ldg(&F[3 * f + 1]);
    ids[3] = __ldg(&F[3 * f + 2]);
  } else {
    vf = false;
    int64_t r = q - n_vf;
    int a = __ldg(&eep[2 * r]);
    int b = __ldg(&eep[2 * r + 1]);
    ids[0] = __ldg(&E[2 * a]);
    ids[1] = __ldg(&E[2 * a + 1]);
    ids[2] = __ldg(&E[2 * b]);
    ids[3] = __ldg(&E[2 * b + 1]);
  }
}

// Query records (the paper's CD step, Section "Broad-Phase", computed once per
// query in a dense pass, prepare_record): the set-up of setup_query stored as
// structure of arrays with stride rec_stride -- 24 words per query, c0[3][3],
// dc[3][3] (word 3j + x and 9 + 3j + x), the error box e[3] (as a double, word
// 18 + x) and the split keys K[3] (words 21-23; bit 63 of K[0] marks a
// vertex-face query) -- then 33 floats: c0f, dcf of vector j on axis x at
// 2 (3j + x) and 2 (3j + x) + 1, and per axis tn, tm, wn, cc0, cdc at
// 18 + 5x ... 22 + 5x.
constexpr int kRecWords = 24;

__device__ __forceinline__ void load_record(QueryData &Q, bool &vf, const unsigned long long *__restrict__ rec,
                                            int64_t stride, int64_t q) {
  int w = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) Q.c0[j][x] = __longlong_as_double((long long)__ldg(&rec[(w++) * stride + q]));
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) Q.dc[j][x] = __longlong_as_double((long long)__ldg(&rec[(w++) * stride + q]));
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const long long e = (long long)__ldg(&rec[(w++) * stride + q]);
    Q.ebox_p[x] = e;
    Q.ebox_n[x] = f64_ord(-__longlong_as_double(e));
  }
  unsigned long long k0 = __ldg(&rec[(w++) * stride + q]);
  vf = (k0 >> 63) != 0;
  Q.K[0] = k0 & ~(1ull << 63);
  Q.K[1] = __ldg(&rec[(w++) * stride + q]);
  Q.K[2] = __ldg(&rec[(w++) * stride + q]);
  const float *r32 = (const float *)(rec + kRecWords * stride);
  int f = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Q.c0f[j][x] = __ldg(&r32[(f++) * stride + q]);
      Q.dcf[j][x] = __ldg(&r32[(f++) * stride + q]);
    }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Q.tn[x] = __ldg(&r32[(f++) * stride + q]);
    Q.tm[x] = __ldg(&r32[(f++) * stride + q]);
    Q.wn[x] = __ldg(&r32[(f++) * stride + q]);
    Q.cc0[x] = __ldg(&r32[(f++) * stride + q]);
    Q.cdc[x] = __ldg(&r32[(f++) * stride + q]);
  }
}

// Staged queries: a warp claims kStageQ consecutive queries at a time and
// copies their records into shared memory with cp.async one batch ahead, so
// that neither the claim (an L2 atomic) nor the record (DRAM) is waited on
// when lanes take new queries.
constexpr int kRecFloats = 33;
struct __align__(16) Stage {
  unsigned long long w[kRecWords][kStageQ];
  float f[kRecFloats][kStageQ];
  int sid[kStageQ];
};
static_assert(sizeof(Stage) == kStageBytes, "stage layout");

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
  const size_t ga = __cvta_generic_to_global(gmem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(ga) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

// Copy the records of queries [b, b + kStageQ) into S (one commit group per
// lane).  b is a multiple of kStageQ and the record arrays hold a multiple of
// kStageQ entries, so every 16-byte chunk is aligned and in bounds.
__device__ __forceinline__ void stage_copy(Stage &S, const NarrowArgs &A, unsigned long long b, int lane) {
  constexpr int kW = kRecWords * kStageQ / 2;     // 16-byte chunks of the words
  constexpr int kF = kRecFloats * kStageQ / 4;    // of the floats
  constexpr int kS = kStageQ / 4;                 // of the scene ids
  const float *r32 = (const float *)(A.qrec + kRecWords * A.rec_stride);
  const int total = kW + kF + (A.mode == 2 ? kS : 0);
  for (int c = lane; c < total; c += 32) {
    if (c < kW) {
      const int w = c / (kStageQ / 2), p = c % (kStageQ / 2);
      cp_async16(&S.w[w][2 * p], A.qrec + w * A.rec_stride + b + 2 * p);
    } else if (c < kW + kF) {
      const int f = (c - kW) / (kStageQ / 4), p = (c - kW) % (kStageQ / 4);
      cp_async16(&S.f[f][4 * p], r32 + f * A.rec_stride + b + 4 * p);
    } else {
      const int p = c - kW - kF;
      cp_async16(&S.sid[4 * p], A.qsid + b + 4 * p);
    }
  }
  cp_async_commit();
}

__device__ __forceinline__ void load_record_stage(QueryData &Q, bool &vf, const Stage &S, int i) {
  int w = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) Q.c0[j][x] = __longlong_as_double((long long)S.w[w++][i]);
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) Q.dc[j][x] = __longlong_as_double((long long)S.w[w++][i]);
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    const long long e = (long long)S.w[w++][i];
    Q.ebox_p[x] = e;
    Q.ebox_n[x] = f64_ord(-__longlong_as_double(e));
  }
  const unsigned long long k0 = S.w[w++][i];
  vf = (k0 >> 63) != 0;
  Q.K[0] = k0 & ~(1ull << 63);
  Q.K[1] = S.w[w++][i];
  Q.K[2] = S.w[w++][i];
  int f = 0;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int x = 0; x < 3; ++x) {
      Q.c0f[j][x] = S.f[f++][i];
      Q.dcf[j][x] = S.f[f++][i];
    }
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    Q.tn[x] = S.f[f++][i];
    Q.tm[x] = S.f[f++][i];
    Q.wn[x] = S.f[f++][i];
    Q.cc0[x] = S.f[f++][i];
    Q.cdc[x] = S.f[f++][i];
  }
}

}  // namespace

// Block queue (tail phase): a warp whose lanes all carry work hands its
// lanes' shallowest owed siblings to the idle warps of its own block through
// shared memory, so that a long query spreads over the block's four warps
// without any L2 round trip on the busy warp (the device-wide ring, for
// other blocks, costs several).  A cell at position p holds a unit when
// seq == p + 1 and is free for position p + kBQ once its taker stores
// seq = p + kBQ.  `local` counts the units handed out this way and not yet
// finished (in the queue or in a lane); they are not in the device-wide
// `pending` count, so a warp leaves only when its block's count is zero too.
constexpr int kBQ = 64;                  // cells of a block's queue
constexpr unsigned long long kBQMax = 32;   // units queued at most
struct BlockQueue {
  unsigned long long seq[kBQ];
  unsigned long long w[kBQ][3];          // t, u, v: numerator | level << 54
  uint32_t q[kBQ];
  unsigned long long head, tail;         // positions, monotonic
  int idle;                              // warps of the block that have no work
  int local;                             // units handed out through the queue, not finished
};

__device__ __forceinline__ unsigned long long vload(const unsigned long long *p) {
  return *(const volatile unsigned long long *)p;
}

// Branches the bulk of the launch rarely takes (the tail's work sharing,
// idling, the iteration and level caps, the full FP64 evaluation, paths
// deeper than the masks): hinted, so that the common path stays contiguous
// in the instruction cache.
#ifndef CCD_NO_HINTS
#define CCD_COLD(c) __builtin_expect(!!(c), 0)
#else
#define CCD_COLD(c) (c)
#endif

constexpr int kIdleRounds = 1 << 14;   // idle warp rounds before a warp retires
// idle back-off bounds (ns): warps polling the ring more often than this
// slow the busy warps of the tail (measured: 0.25-2 us worse, 1-32 us best)
constexpr unsigned kNapMin = 1000, kNapMax = 32000;
constexpr int kRefresh = 8;            // iterations between reads of the shared values
constexpr int kDonateMin = 4;          // idle lanes a warp gathers before a round of donation
// A query whose work is split over several units (donation, hand-off) shares
// one iteration budget: each unit counts its evaluations in windows of at
// most kBudgetWindow and adds them to the query's counter at the end of each
// window, where it also learns whether the query has passed max_iter.  A
// query kept by one lane counts privately and is capped exactly at max_iter.
constexpr long long kBudgetWindow = 64;

// End of a budget window of a unit of a split query (cnt = cap_left + 1: the
// evaluation about to run is the first past the window): add the window's
// evaluations to the query's counter; if the query is still within max_iter,
// open the next window with this evaluation counted and return true.  A unit
// that owns its whole query has no windows (its budget is max_iter itself).
__device__ __forceinline__ bool next_budget_window(const NarrowArgs &A, int64_t q, bool whole, long long &cnt,
                                                   long long &cap_left) {
  if (whole) return false;
  const unsigned long long done = (unsigned long long)(cnt - 1);
  const unsigned long long tot = atomicAdd(&A.qiters[q], done) + done;
  if (tot < (unsigned long long)A.max_iter) {
    cnt = 1;
    cap_left = min(kBudgetWindow, A.max_iter - (long long)tot);
    return true;
  }
  cnt = 1;   // flushed; the cap path below takes the attempted evaluation back out
  return false;
}

// Control flow is warp-uniform at the loop level: refill, idling and exit are
// decided for the whole warp (ballots and broadcasts), and the per-lane work
// sits in structured branches, so the lanes of a warp reconverge every
// iteration and the FP64 instructions of an interval issue once per warp.
template <bool kRecords>
__device__ __forceinline__ void narrow_body(NarrowArgs A) {
  DevCtl *ctl = A.ctl;
  if (A.only_if_rerun && ctl->rerun == 0) return;
  if (A.counts_from_ctl) {
    A.n_vf = ctl->pair_counts[0];
    A.n_ee = ctl->pair_counts[1];
    if (A.ee_end > 0) A.ee = A.vf + 2 * (A.ee_end - A.n_ee);
  }
  const unsigned FULL = 0xFFFFFFFFu;
  const int64_t nq = A.n_vf + A.n_ee;
  const int lane = threadIdx.x & 31;
  const unsigned lt_mask = (1u << lane) - 1u;
  const unsigned long long delta_bits = dbits(A.delta);
  const unsigned long long ring_cap = A.ring_mask + 1;

  __shared__ SharedQuery SQ;                 // FP64 part of each lane's query
  __shared__ BlockQueue BQ;
  const int tid = threadIdx.x;
  if (tid == 0) {
    BQ.head = BQ.tail = 0;
    BQ.idle = 0;
    BQ.local = 0;
  }
  for (int i = tid; i < kBQ; i += blockDim.x) BQ.seq[i] = (unsigned long long)i;
  __syncthreads();
  // single-precision filter data and split keys of the lane's query
  float c0f[3][3], dcf[3][3], tn[3], tm[3], wn[3];
  unsigned long long K[3] = {0, 0, 0};
  bool vf = false;
  __shared__ int SID[kNarrowThreads];        // mode 2: scene of the lane's query
  // mode 2: the t* of the lane's scene in use (row 0) and loaded one refresh
  // ahead (row 1)
  __shared__ unsigned long long SCN[2][kNarrowThreads];
  SCN[0][tid] = SCN[1][tid] = kInfBits;
  bool have = false, fresh = false, whole = false;
  bool blocal = false;                       // the unit came through the block queue
  bool widle = false;                        // warp-uniform: counted in BQ.idle
  bool exhausted = false;                    // warp-uniform
  int64_t q = -1;   // the query whose data the lane's registers and shared column hold (-1: none yet)
  Node N{0, 0, 0, 0, 0, 0};
  int depth = 0, root_depth = 0;
  // the path as bit masks over the 31 depths below rb, the depth at which
  // the lane took its unit (0 for a whole query): pend bit d is set while the
  // path node at depth rb + d is a left child whose right sibling is still
  // owed, and bit d of (axhi, axlo) is the axis that was split to reach depth
  // rb + d; a unit that goes deeper (`deep`) backtracks by walking the path
  // instead.  (The long queries of a scene do most of their work 32-37
  // levels down; the pieces other lanes take from them start well below
  // the root, so with masks counted from their own start they stay on the
  // mask path.)
  unsigned pend = 0, axlo = 0, axhi = 0;
  int rb = 0;
  // bit d of tright: the path node at depth rb + d is the right child of a
  // split along t (the path's t_lo grows exactly at those depths)
  unsigned tright = 0;
  bool deep = false;
  unsigned long long tq = kInfBits;          // bits of this unit's best t*
  long long cnt = 0, cap_left = 0;
  unsigned flags = 0;
  unsigned n_eval = 0, n_eval64 = 0;          // per lane, per launch
  int idle_rounds = 0;                       // warp-uniform: idle rounds in a row
  int bq_polls = 0;                          // warp-uniform: block-queue polls since the last round
  unsigned ended_acc = 0;                    // warp-uniform: ended units not yet subtracted from pending
  // Shared values (global t*, next query, the scene's t*) are read from L2
  // every kRefresh iterations into a second slot and used from the first,
  // so that no iteration waits for an L2 round trip; stale values only prune
  // less or hand work out later.  Warp-uniform state that is touched only
  // at claims, refreshes, hand-offs and the end (lane 0 writes it, behind
  // __syncwarp) lives in shared memory, not in registers: the loop then
  // needs fewer registers than 3 blocks of 128 threads allow, spill-free.
  struct WarpCtl {
    unsigned long long pf_toi, pf_qnext, nx_toi, nx_qnext, pf_occ, nx_head, nx_tail;
    unsigned long long c_reg;                 // lane 0's claim after the next batch
    uint32_t s_base, n_base;                  // staged batches (query indices < 2^32)
    int sbuf, s_n, s_pos, n_n, claims_done;
    unsigned n_exp, n_cap, n_don, n_eval_tail;
    long long wsince;                         // evaluations in the tail since the last hand-off
  };
  __shared__ WarpCtl WC[kNarrowThreads / 32];
  WarpCtl &wc = WC[threadIdx.x >> 5];
  if (lane == 0) {
    wc.pf_toi = kInfBits;
    wc.pf_qnext = 0;
    wc.pf_occ = 0;
    wc.n_exp = wc.n_cap = wc.n_don = wc.n_eval_tail = 0;
    wc.wsince = 0;
  }
  unsigned long long g_toi = kInfBits;                          // all lanes: pf_toi at the last refresh
  bool g_tail = false;                                          // all lanes: every query taken (last refresh)
  unsigned long long cut_prev = ~0ull;                          // cut53 = ceil53(cut_prev)
  uint64_t cut53 = 0;
  int pf_age = 0;
  if (lane == 0) {
    wc.nx_toi = ld_relaxed_u64(&ctl->toi_bits);
    wc.nx_qnext = ld_relaxed_u64(&ctl->q_next);
    wc.nx_head = ld_relaxed_u64(&ctl->q_head);
    wc.nx_tail = ld_relaxed_u64(&ctl->q_tail);
  }
  __syncwarp(FULL);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicCAS(&ctl->t_start, 0ull, globaltimer());

  // Staged claims (with query records only): the current batch [s_base,
  // s_base + s_n) of which s_pos are taken, the next batch (records in
  // flight into the other buffer) and the claim after it (WarpCtl).
  extern __shared__ __align__(16) unsigned char dyn_smem[];
#define ST ((Stage *)dyn_smem + 2 * (threadIdx.x >> 5))
  const bool staged = kRecords;
  if (staged) {
    unsigned long long b0 = 0, b1 = 0;
    if (lane == 0) {
      b0 = atomicAdd(&ctl->q_next, (unsigned long long)kStageQ);
      b1 = atomicAdd(&ctl->q_next, (unsigned long long)kStageQ);
      wc.c_reg = atomicAdd(&ctl->q_next, (unsigned long long)kStageQ);
    }
    b0 = __shfl_sync(FULL, b0, 0);
    b1 = __shfl_sync(FULL, b1, 0);
    const unsigned long long un = (unsigned long long)nq;
    const int s_n = b0 < un ? (int)min((unsigned long long)kStageQ, un - b0) : 0;
    const int n_n = b1 < un ? (int)min((unsigned long long)kStageQ, un - b1) : 0;
    const bool claims_done = n_n < kStageQ;
    if (lane == 0) {
      wc.s_base = (uint32_t)b0;
      wc.s_n = s_n;
      wc.n_base = (uint32_t)b1;
      wc.n_n = n_n;
      wc.claims_done = claims_done;
      wc.sbuf = 0;
      wc.s_pos = 0;
    }
    if (lane == 0 && s_n + n_n > 0) atomicAdd(&ctl->pending, (unsigned long long)(s_n + n_n));
    if (s_n > 0) stage_copy(ST[0], A, b0, lane);
    if (n_n > 0) stage_copy(ST[1], A, b1, lane);
    cp_async_wait_1();   // the first batch (the second may still be in flight)
    if (n_n == 0) cp_async_wait_all();
    __syncwarp(FULL);
    if (claims_done && lane == 0 && ld_relaxed_u64(&ctl->t_exhausted) == 0)
      atomicCAS(&ctl->t_exhausted, 0ull, globaltimer());
  }

  while (true) {
    int slot = -1;   // stage slot of a query taken in this iteration
    // ---- 1. refill lanes without work: queries, then exported intervals --
    // (intervals are exported only once every query has been handed out,
    // so a warp looks at the ring only after its own claim came back empty)
    if (__any_sync(FULL, !have)) {
      const unsigned long long pf_toi_b = g_toi;
      const unsigned m = __ballot_sync(FULL, !have);
      if (m && !exhausted && staged) {
        // the warp's staging state, kept in shared memory between claims
        int sbuf = wc.sbuf, s_n = wc.s_n, s_pos = wc.s_pos, n_n = wc.n_n;
        uint32_t s_base = wc.s_base, n_base = wc.n_base;
        bool claims_done = wc.claims_done;
        if (s_pos == s_n) {
          if (n_n == 0) {
            exhausted = true;
          } else {
            // start the next batch (copied one swap ago) and copy the batch
            // claimed one swap ago into the buffer just emptied
            cp_async_wait_all();
            __syncwarp(FULL);
            sbuf ^= 1;
            s_base = n_base;
            s_n = n_n;
            s_pos = 0;
            n_n = 0;
            if (!claims_done) {
              const unsigned long long nb = wc.c_reg;
              const int nn = nb < (unsigned long long)nq ? (int)min((unsigned long long)kStageQ,
                                                                    (unsigned long long)nq - nb) : 0;
              claims_done = nn < kStageQ;
              if (nn > 0) {
                n_base = (uint32_t)nb;
                n_n = nn;
                stage_copy(ST[sbuf ^ 1], A, nb, lane);
                if (lane == 0) atomicAdd(&ctl->pending, (unsigned long long)nn);
              }
              __syncwarp(FULL);   // every lane has read c_reg
              if (!claims_done && lane == 0) wc.c_reg = atomicAdd(&ctl->q_next, (unsigned long long)kStageQ);
              if (claims_done && lane == 0 && ld_relaxed_u64(&ctl->t_exhausted) == 0)
                atomicCAS(&ctl->t_exhausted, 0ull, globaltimer());
            }
          }
        }
        if (s_pos < s_n) {
          const int k = min(__popc(m), s_n - s_pos);
          const int rank = __popc(m & lt_mask);
          if (!have && rank < k) {
            slot = s_pos + rank;
            q = (int64_t)s_base + slot;
            have = fresh = whole = true;
            N = Node{0, 0, 0, 0, 0, 0};
          }
          s_pos += k;
        }
        __syncwarp(FULL);   // every lane has read the staging state
        if (lane == 0) {
          wc.sbuf = sbuf;
          wc.s_n = s_n;
          wc.s_pos = s_pos;
          wc.n_n = n_n;
          wc.s_base = s_base;
          wc.n_base = n_base;
          wc.claims_done = claims_done;
        }
        __syncwarp(FULL);
      } else if (m && !exhausted) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&ctl->q_next, (unsigned long long)__popc(m));
        base = __shfl_sync(FULL, base, 0);
        if (base + __popc(m) >= (unsigned long long)nq) {
          exhausted = true;
          if (lane == 0 && ld_relaxed_u64(&ctl->t_exhausted) == 0)
            atomicCAS(&ctl->t_exhausted, 0ull, globaltimer());
        }
        if (!have) {
          const unsigned long long mine = base + __popc(m & lt_mask);
          if ((int64_t)mine < nq) {
            q = (int64_t)mine;
            have = fresh = whole = true;
            N = Node{0, 0, 0, 0, 0, 0};
          }
        }
        const int got = base < (unsigned long long)nq
                            ? (int)min((unsigned long long)__popc(m), (unsigned long long)nq - base)
                            : 0;
        if (lane == 0 && got) atomicAdd(&ctl->pending, (unsigned long long)got);
      }
      // A warp with no work at all takes first from its block's queue (up to
      // one cell per lane: lanes test the cells' sequence numbers, lane 0
      // claims the ready prefix with one shared-memory CAS).
      if (CCD_COLD(exhausted && __ballot_sync(FULL, have) == 0)) {
        unsigned long long h = 0;
        if (lane == 0) h = vload(&BQ.head);
        h = __shfl_sync(FULL, h, 0);
        const bool ready = vload(&BQ.seq[(h + lane) % kBQ]) == h + lane + 1;
        const unsigned rb = __ballot_sync(FULL, ready);
        const int r = rb == FULL ? 32 : __ffs(~rb) - 1;
        int ok = 0;
        if (r > 0 && lane == 0) ok = atomicCAS(&BQ.head, h, h + r) == h;
        ok = __shfl_sync(FULL, ok, 0);
        if (ok && lane < r) {
          const int cell = (int)((h + lane) % kBQ);
          __threadfence_block();   // the cell's contents after its sequence number
          const unsigned long long w0 = BQ.w[cell][0], w1 = BQ.w[cell][1], w2 = BQ.w[cell][2];
          const unsigned long long m54 = (1ull << 54) - 1;
          q = BQ.q[cell];
          N.n0 = w0 & m54;
          N.n1 = w1 & m54;
          N.n2 = w2 & m54;
          N.l0 = (int)(w0 >> 54);
          N.l1 = (int)(w1 >> 54);
          N.l2 = (int)(w2 >> 54);
          __threadfence_block();   // read before the cell is freed
          *(volatile unsigned long long *)&BQ.seq[cell] = h + lane + kBQ;
          have = fresh = true;
          whole = false;
          blocal = true;
        }
      }
      // Only a warp with no work at all takes from the ring: a warp with busy
      // lanes fills its idle ones by donation below (shuffles and shared
      // memory), which costs none of the ring's L2 round trips that would
      // otherwise sit on the path of the tail's long queries.
      if (CCD_COLD(exhausted && __ballot_sync(FULL, have) == 0 && wc.pf_occ > 0)) {
        // pop up to one cell per idle lane: lanes test the cells' sequence
        // numbers in parallel, lane 0 claims the ready prefix with one CAS
        const unsigned m = __ballot_sync(FULL, !have);
        const int want = __popc(m);
        unsigned long long h = 0;
        if (lane == 0) h = ld_relaxed_u64(&ctl->q_head);
        h = __shfl_sync(FULL, h, 0);
        const bool ready = lane < want && ld_acquire_u64(&A.ring[(h + lane) & A.ring_mask].seq) == h + lane + 1;
        const unsigned rb = __ballot_sync(FULL, ready);
        const int r = rb == FULL ? 32 : __ffs(~rb) - 1;
        int ok = 0;
        if (r > 0 && lane == 0) ok = atomicCAS(&ctl->q_head, h, h + r) == h;
        ok = __shfl_sync(FULL, ok, 0);
        const int rank = __popc(m & lt_mask);
        if (ok && !have && rank < r) {
          const unsigned long long pos = h + rank;
          RingCell *c = &A.ring[pos & A.ring_mask];
          (void)ld_acquire_u64(&c->seq);   // pairs with the writer's release
          const unsigned long long w0 = c->w[0], w1 = c->w[1], w2 = c->w[2];
          const unsigned long long m54 = (1ull << 54) - 1;
          q = c->q;
          N.n0 = w0 & m54;
          N.n1 = w1 & m54;
          N.n2 = w2 & m54;
          N.l0 = (int)(w0 >> 54);
          N.l1 = (int)(w1 >> 54);
          N.l2 = (int)(w2 >> 54);
          st_release_u64(&c->seq, pos + A.ring_mask + 1);   // free for the next lap
          have = fresh = true;
          whole = false;
          blocal = false;
        }
      }
      // Intra-warp donation: lanes still idle (no query left; the ring is for
      // idle warps) take the shallowest pending sibling of a busy lane of their
      // own warp; the query data moves by shuffles, the donor keeps the rest
      // of its subtree (its root moves down to the donated sibling's depth).
      const unsigned idle = __ballot_sync(FULL, !have);
      if (CCD_COLD(exhausted && __popc(idle) >= kDonateMin)) {
        // candidate donors: the first busy lanes, one per idle lane; only they
        // walk their path to find the shallowest pending sibling
        const unsigned busy = __ballot_sync(FULL, have && !fresh);
        const bool cand = have && !fresh && __popc(busy & lt_mask) < __popc(idle);
        Node S{0, 0, 0, 0, 0, 0};
        int dS = 0;
        if (cand) {
          unsigned long long c = tq;
          if (A.mode == 1) c = min(c, pf_toi_b);
          if (A.mode == 2) c = min(c, SCN[0][tid]);
          if (deep) {
            dS = shallowest_pending(K, N, depth, root_depth, c, S);
          } else {
            const int d = shallowest_owed(N, depth - rb, root_depth - rb, pend, axlo, axhi, c, S);
            dS = d > 0 ? rb + d : 0;
          }
        }
        const unsigned donors = __ballot_sync(FULL, dS > 0);
        const int pairs = min(__popc(donors), __popc(idle));
        if (pairs > 0) {
          // every donated subtree is a new unit for the termination count
          if (lane == 0) atomicAdd(&ctl->pending, (unsigned long long)pairs);
          const bool recv = !have && __popc(idle & lt_mask) < pairs;
          const bool give = dS > 0 && __popc(donors & lt_mask) < pairs;
          const int src = recv ? (int)__fns(donors, 0, __popc(idle & lt_mask) + 1) : lane;
          const long long qv = __shfl_sync(FULL, (long long)q, src);
          // A receiver whose last unit was a piece of the same query still
          // holds that query's data in its registers and shared column (the
          // data depend on the query only).  In the tail the lanes of a warp
          // mostly share one long query, so the data move only when some
          // receiver holds another query.
          const bool move = recv && qv != q;
          __syncwarp(FULL);
          if (__any_sync(FULL, move)) {
            if (move) copy_shared(SQ, tid, (tid & ~31) | src);   // the donor's FP64 data
#pragma unroll
            for (int j = 0; j < 3; ++j)
#pragma unroll
              for (int x = 0; x < 3; ++x) {
                const float a = __shfl_sync(FULL, c0f[j][x], src);
                const float b = __shfl_sync(FULL, dcf[j][x], src);
                if (move) {
                  c0f[j][x] = a;
                  dcf[j][x] = b;
                }
              }
#pragma unroll
            for (int x = 0; x < 3; ++x) {
              const float a = __shfl_sync(FULL, tn[x], src);
              const float b = __shfl_sync(FULL, tm[x], src);
              const float c = __shfl_sync(FULL, wn[x], src);
              const unsigned long long kk = __shfl_sync(FULL, K[x], src);
              if (move) {
                tn[x] = a;
                tm[x] = b;
                wn[x] = c;
                K[x] = kk;
              }
            }
            const int sidv = A.mode == 2 ? SID[(tid & ~31) + src] : 0;   // (a busy lane's entry)
            const int vfv = __shfl_sync(FULL, (int)vf, src);
            if (move) {
              if (A.mode == 2) SID[tid] = sidv;
              vf = vfv != 0;
            }
          }
          const uint64_t s0 = __shfl_sync(FULL, S.n0, src), s1 = __shfl_sync(FULL, S.n1, src),
                         s2 = __shfl_sync(FULL, S.n2, src);
          const int l0 = __shfl_sync(FULL, S.l0, src), l1 = __shfl_sync(FULL, S.l1, src),
                    l2 = __shfl_sync(FULL, S.l2, src);
          const unsigned long long tqv = __shfl_sync(FULL, tq, src);

          if (recv) {
            q = qv;
            SCN[0][tid] = SCN[1][tid] = kInfBits;
            N = Node{s0, s1, s2, l0, l1, l2};
            depth = root_depth = rb = N.depth();
            pend = tright = 0;
            deep = false;
            tq = tqv;
            cap_left = min(kBudgetWindow, A.max_iter);   // the query's shared budget, in windows
            cnt = 0;
            flags = 0;
            have = true;
            whole = false;
            blocal = false;
          }
          if (give) {
            root_depth = dS;   // the donated sibling is no longer ours
            atomicAdd(&wc.n_don, 1u);
            if (whole) {
              // the query's budget becomes shared: publish the evaluations so
              // far (the counter was 0 while this lane owned the query)
              atomicAdd(&A.qiters[q], (unsigned long long)cnt);
              cap_left = min(kBudgetWindow, cap_left - cnt);
              cnt = 0;
              whole = false;
            }
          }
        }
      }
    }

    // ---- 2. a warp with no work idles or retires (uniform) ----------------
    if (CCD_COLD(__ballot_sync(FULL, have) == 0)) {
      if (ended_acc) {
        if (lane == 0) atomicAdd(&ctl->pending, (unsigned long long)(-(long long)ended_acc));
        ended_acc = 0;
        __threadfence();
      }
      if (!widle) {
        if (lane == 0) atomicAdd(&BQ.idle, 1);
        widle = true;
      }
      // While a warp of the block still works (it may queue units), poll the
      // block's queue every kNapMin (at once while it holds units) and the
      // device-wide state every 32 polls; otherwise back off, kNapMin
      // doubling up to kNapMax.
      const bool items = exhausted && vload(&BQ.tail) != vload(&BQ.head);
      const bool mates_busy = *(volatile int *)&BQ.idle < (int)(blockDim.x >> 5);
      if ((items || mates_busy) && ++bq_polls < 32) {
        if (!items) __nanosleep(kNapMin);
        continue;
      }
      bq_polls = 0;
      int stop = 0;
      if (lane == 0) {
        const unsigned long long h = ld_relaxed_u64(&ctl->q_head), t = ld_relaxed_u64(&ctl->q_tail);
        const unsigned long long pend = ld_relaxed_u64(&ctl->pending);
        wc.pf_occ = t > h ? t - h : 0;   // an idle warp sees new exports at once
        stop = (exhausted && wc.pf_occ == 0 && pend == 0 && *(volatile int *)&BQ.local == 0) ||
               idle_rounds >= kIdleRounds;
      }
      if (__shfl_sync(FULL, stop, 0)) {
        if (lane == 0) atomicSub(&BQ.idle, 1);   // (no longer there to take units)
        break;
      }
      __nanosleep(mates_busy ? kNapMin : min(kNapMin << min(idle_rounds, 5), kNapMax));
      ++idle_rounds;   // (while a block mate works: one round per 32 polls of the block's queue)
      continue;
    }
    idle_rounds = 0;
    bq_polls = 0;
    if (widle) {
      if (lane == 0) atomicSub(&BQ.idle, 1);
      widle = false;
    }

    // ---- 3. set up newly acquired units ------------------------------------
    if (fresh) {
      QueryData Q;
      if constexpr (kRecords) {
        if (slot >= 0) {
          load_record_stage(Q, vf, ST[wc.sbuf], slot);
          if (A.mode == 2) SID[tid] = ST[wc.sbuf].sid[slot];
        } else {
          load_record(Q, vf, A.qrec, A.rec_stride, q);
          if (A.mode == 2) SID[tid] = A.qsid[q];
        }
      } else {
        int ids[4];
        query_ids(q, A.n_vf, A.vf, A.ee, A.E, A.F, ids, vf);
        setup_query(Q, vf, ids, A.V0, A.V1, A.nV, A.min_sep, A.delta);
        if (A.mode == 2) SID[tid] = A.qsid[q];
      }
      put_shared(SQ, tid, Q);
      SCN[0][tid] = SCN[1][tid] = kInfBits;   // the loaded values belonged to the previous query
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          c0f[j][x] = Q.c0f[j][x];
          dcf[j][x] = Q.dcf[j][x];
        }
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        tn[x] = Q.tn[x];
        tm[x] = Q.tm[x];
        wn[x] = Q.wn[x];
        K[x] = Q.K[x];
      }
      depth = root_depth = rb = N.depth();
      pend = tright = 0;
      deep = false;
      cnt = 0;
      flags = 0;
      tq = kInfBits;
      cap_left = A.max_iter;
      if (whole) {
        // the lane that takes a query owns its slots until it hands work out
        A.qflags[q] = 0;
        A.qiters[q] = 0;
        if (A.mode == 0) {
          if (q < A.n_vf) A.toi_vf_bits[q] = kInfBits;
          else A.toi_ee_bits[q - A.n_vf] = kInfBits;
        }
      } else {
        if (A.mode == 0) tq = ld_relaxed_u64(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf]);
        const long long used = (long long)ld_relaxed_u64(&A.qiters[q]);
        cap_left = used >= A.max_iter ? 0 : min(kBudgetWindow, A.max_iter - used);
      }
      fresh = false;
    }

    // ---- 4. ProcessInterval on the current node ---------------------------
    // shared values loaded during the previous iteration (stale values only
    // prune less or hand off later)
    if (CCD_COLD(++pf_age == kRefresh)) {
      pf_age = 0;
      if (lane == 0) {
        wc.pf_toi = wc.nx_toi;
        wc.pf_qnext = wc.nx_qnext;
        wc.pf_occ = wc.nx_tail > wc.nx_head ? wc.nx_tail - wc.nx_head : 0;
        if (wc.pf_occ > 0) atomicMax(&ctl->queue_peak, wc.pf_occ);
        wc.nx_toi = ld_relaxed_u64(&ctl->toi_bits);
        wc.nx_qnext = ld_relaxed_u64(&ctl->q_next);
        wc.nx_head = ld_relaxed_u64(&ctl->q_head);
        wc.nx_tail = ld_relaxed_u64(&ctl->q_tail);
      }
      __syncwarp(FULL);
      if (A.mode == 2) {
        SCN[0][tid] = SCN[1][tid];
        if (have) SCN[1][tid] = ld_relaxed_u64(&A.toi_scene[SID[tid]]);
      }
      // broadcast once per refresh, not per iteration
      g_toi = wc.pf_toi;
      g_tail = wc.pf_qnext >= (unsigned long long)nq;
    }
    unsigned long long cut = tq;
    const unsigned long long g = g_toi;
    // hand work out only once every query has been taken (idle lanes exist)
    const bool tail_phase = g_tail;
    if (A.mode == 1) cut = g < cut ? g : cut;
    if (A.mode == 2) cut = min(SCN[0][tid], cut);
    bool node_done = true;     // false when the node was split (go to its left child)
    bool unit_end = false;
    bool evaluate = false;
    if (cut != cut_prev) {     // (t* changes rarely)
      cut_prev = cut;
      cut53 = ceil53(cut);
    }
    if (have) {
      if (s53(N.n0, N.l0) >= cut53) {
        // pruned: starts at or after the current t*
      } else if (vf && outside_simplex(N)) {
        // vertex-face: u_lo > 1 - v_lo, the interval lies outside the simplex
      } else if (CCD_COLD(!(A.no_zero && N.n0 == 0) && ++cnt > cap_left &&
                          !next_budget_window(A, q, whole, cnt, cap_left))) {
        // iteration cap: t* = min(t*, earliest left end among the live intervals)
        unsigned long long m = dbits(dyadic(N.n0, N.l0));
        Node W = N;
        for (int d = depth; d > root_depth; --d) {
          int a = last_axis(K, W);
          if ((W.n(a) & 1) == 0) {
            unsigned long long sb = dbits(a == 0 ? dyadic(W.n0 + 1, W.l0) : dyadic(W.n0, W.l0));
            m = sb < m ? sb : m;
          }
          W.up(a);
        }
        tq = m < tq ? m : tq;
        if (A.mode == 1) atomicMin(&ctl->toi_bits, tq);       // (modes 1, 2: as an accept)
        if (A.mode == 2) atomicMin(&A.toi_scene[SID[tid]], tq);
        flags |= CCD_FLAG_ITER_CAP;
        atomicAdd(&wc.n_cap, 1u);
        --cnt;
        unit_end = true;
      } else {
        evaluate = true;
      }
    }
    if (evaluate) {
      ++n_eval;
      // Single-precision filter: when every level is <= 24 the interval's
      // ends are exact floats and the FP32 hull is within e32 of the FP64
      // hull, its certified ends L, H bound R's; a miss, or a split (no miss,
      // not narrow, not inside), proven on it is certainly the FP64 decision,
      // so FP64 runs only on the rest.
      bool decided = false, miss = false, accept = false;
      bool full = true;            // the full FP64 evaluation decides
      unsigned need = 0, tb = 0;   // ends FP32 left open: bit x low, bit 3 + x high
      if (max(max(N.l0, N.l1), N.l2) <= 24) {
        Box3f Bf;
        float cc0[3], cdc[3];
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          cc0[x] = SQ.cc0[x][tid];
          cdc[x] = SQ.cdc[x][tid];
        }
        inclusion32(c0f, dcf, cc0, cdc, vf, dyadic32(N.n0, N.l0), dyadic32(N.n0 + 1, N.l0), dyadic32(N.n1, N.l1),
                    dyadic32(N.n1 + 1, N.l1), dyadic32(N.n2, N.l2), dyadic32(N.n2 + 1, N.l2), Bf);
        // (levels <= 24 here: the corner checks below take their ends as
        // exact doubles from these floats)
        bool cmiss = false, cni = false, cnn = false;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          cmiss |= (Bf.lo[x] > tm[x]) | (Bf.hi[x] < -tm[x]);
          need |= (Bf.L[x] <= tn[x] ? 0u : 1u << x) | (Bf.H[x] >= -tn[x] ? 0u : 8u << x);
          cni |= (Bf.lo[x] < -tm[x]) | (Bf.hi[x] > tm[x]);
          cnn |= __fsub_rn(Bf.hi[x], Bf.lo[x]) >= wn[x];
        }
        tb = Bf.tb;
        if (cmiss) {
          decided = miss = true;
        } else if (cni & cnn) {
          full = false;
          decided = need == 0;   // split
        }
      }
      // Not narrow and not inside, and "no miss" settled on every end but a
      // few: each remaining end is checked on one FP64 corner, the one the FP64
      // hull selects at the t end tb names, computed with the FP64 hull's own
      // operations.  The FP64 low end is the smaller of its two
      // t ends, so a low corner at or below e means no miss on that side, as
      // the full evaluation would find; likewise a high corner at or above -e.
      // An end the corner leaves open goes to the full FP64 evaluation.
      if (!decided && !full) {
        const double ul = f2d_exact(dyadic32(N.n1, N.l1)), ur = f2d_exact(dyadic32(N.n1 + 1, N.l1));
        const double vl = f2d_exact(dyadic32(N.n2, N.l2)), vr = f2d_exact(dyadic32(N.n2 + 1, N.l2));
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          if (need & (9u << x)) {
            const bool nlo = (need >> x) & 1u, nhi = (need >> (3 + x)) & 1u;
            double w = SQ.c0[x][tid], a = SQ.c0[3 + x][tid], b = SQ.c0[6 + x][tid];
            const double dw = SQ.dc[x][tid], da = SQ.dc[3 + x][tid], db = SQ.dc[6 + x][tid];
            // an axis with no motion: fma(t, 0, c) is c (up to the sign of a
            // zero, which neither the selection nor the ordered keys see)
            if (((__double_as_longlong(dw) | __double_as_longlong(da) | __double_as_longlong(db)) << 1) != 0) {
              const bool at_r = nlo ? ((tb >> x) & 1u) : ((tb >> (3 + x)) & 1u);
              const double tt = f2d_exact(dyadic32(N.n0 + (at_r ? 1 : 0), N.l0));
              w = fma(tt, dw, w);
              a = fma(tt, da, a);
              b = fma(tt, db, b);
            }
            const bool ap = __double_as_longlong(a) > 0;
            const bool bp = __double_as_longlong(b) > 0;
            if (nlo) {
              const double fmin = vf ? fma(-(ap ? ur : ul), a, fma(-(bp ? vr : vl), b, w))
                                     : fma(-(bp ? vr : vl), b, fma(ap ? ul : ur, a, w));
              if (f64_ord(fmin) <= SQ.ep[x][tid]) need &= ~(1u << x);
            }
            if (nhi) {
              const double fmax = vf ? fma(-(ap ? ul : ur), a, fma(-(bp ? vl : vr), b, w))
                                     : fma(-(bp ? vl : vr), b, fma(ap ? ur : ul, a, w));
              if (f64_ord(fmax) >= SQ.en[x][tid]) need &= ~(8u << x);
            }
          }
        }
        decided = need == 0;   // split
      }
      if (CCD_COLD(!decided)) {
        ++n_eval64;
        const double tr = dyadic(N.n0 + 1, N.l0);
        const double ul = dyadic(N.n1, N.l1), ur = dyadic(N.n1 + 1, N.l1);
        const double vl = dyadic(N.n2, N.l2), vr = dyadic(N.n2 + 1, N.l2);
        Box3 B;
        inclusion_shared(SQ, tid, vf, dyadic(N.n0, N.l0), tr, ul, ur, vl, vr, B);
        bool inside = true, narrow = true;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          const long long lo = f64_ord(B.lo[x]), hi = f64_ord(B.hi[x]);
          const long long ep = SQ.ep[x][tid], en = SQ.en[x][tid];
          miss |= (lo > ep) | (hi < en);
          inside &= (lo >= en) & (hi <= ep);
          narrow &= dbits(__dsub_rn(B.hi[x], B.lo[x])) < delta_bits;
        }
        // zero-TOI rule: an interval starting at t = 0 is always split
        accept = (narrow || inside) && !(A.no_zero && N.n0 == 0);
      }
      if (!miss) {
        int a = -1;
        if (!accept) {
          a = split_axis(K, N);
          if (CCD_COLD(a < 0)) {
            accept = true;
            flags |= CCD_FLAG_LEVEL_CAP;
          }
        }
        if (accept) {
          tq = dbits(dyadic(N.n0, N.l0));
          if (A.mode == 1) atomicMin(&ctl->toi_bits, tq);
          if (A.mode == 2) atomicMin(&A.toi_scene[SID[tid]], tq);
          // Every owed sibling that starts at or after T = this node's t_lo is
          // now pruned; drop them from the path at once instead of visiting
          // them one by one.  A t-sibling starts after T (T lies in its left
          // neighbour); a u- or v-sibling at depth d starts at the t_lo of
          // the path node at depth d - 1, which is below T only if the path
          // went right along t somewhere at depth >= d.
          const int D = tright ? 31 - __clz((int)tright) : 0;
          pend &= (axlo | axhi) & (D >= 31 ? ~0u : (2u << D) - 1u);
        } else {
          N.down_left(a);
          depth += 1;
          node_done = false;
          if (depth - rb < 32) {
            const unsigned bit = 1u << (depth - rb);
            // the right child is owed unless it is already pruned (t* only
            // falls) or lies outside the vertex-face simplex
            bool owe = true;
            if (a == 0) {
              owe = s53(N.n0 + 1, N.l0) < cut53;
            } else if (vf) {
              owe = !(a == 1 ? s53(N.n1 + 1, N.l1) + s53(N.n2, N.l2) > (1ull << 53)
                             : s53(N.n1, N.l1) + s53(N.n2 + 1, N.l2) > (1ull << 53));
            }
            pend = owe ? (pend | bit) : (pend & ~bit);
            tright &= ~bit;
            axlo = (a & 1) ? (axlo | bit) : (axlo & ~bit);
            axhi = (a & 2) ? (axhi | bit) : (axhi & ~bit);
          } else {
            deep = true;
          }
        }
      }
    }

    // ---- 5. next node: backtrack to the deepest pending right sibling ------
    if (have && node_done && !unit_end && !deep) {
      // jump to the deepest owed sibling: undo the splits below it per axis
      // (popcounts of the axis masks), take the right sibling, and go on
      // while the sibling is pruned or outside the simplex
      // (depths relative to rb)
      const int rr = root_depth - rb;
      const unsigned above_root = rr >= 31 ? 0u : ~0u << (rr + 1);
      int dr = depth - rb;
      while (true) {
        const unsigned m = pend & above_root;
        if (m == 0) {
          unit_end = true;
          break;
        }
        const int ds = 31 - __clz((int)m);
        const unsigned r = (dr >= 31 ? ~0u : (2u << dr) - 1u) & (ds >= 31 ? 0u : ~0u << (ds + 1));
        const int c1 = __popc(r & axlo & ~axhi), c2 = __popc(r & axhi);
        const int c0 = dr - ds - c1 - c2;
        N.n0 >>= c0;
        N.l0 -= c0;
        N.n1 >>= c1;
        N.l1 -= c1;
        N.n2 >>= c2;
        N.l2 -= c2;
        const int a = (int)((axlo >> ds) & 1u) | ((int)((axhi >> ds) & 1u) << 1);
        N.add(a, 1);
        dr = ds;
        depth = rb + ds;
        pend &= ~(~0u << ds);
        tright = (tright & ~(~0u << ds)) | (a == 0 ? 1u << ds : 0u);
        const bool pruned = s53(N.n0, N.l0) >= cut53;
        const bool outside = vf && outside_simplex(N);
        if (!pruned && !outside) break;
      }
    } else if (CCD_COLD(have && node_done && !unit_end)) {
      while (true) {
        if (depth == root_depth) {
          unit_end = true;
          break;
        }
        int a = last_axis(K, N);
        if ((N.n(a) & 1) == 0) {
          N.add(a, 1);
          // a right sibling that would be pruned, or that lies outside the
          // vertex-face simplex, is done at once (no iteration spent on it)
          const bool pruned = s53(N.n0, N.l0) >= cut53;
          const bool outside = vf && outside_simplex(N);
          if (!pruned && !outside) break;
        }
        N.up(a);
        depth -= 1;
      }
    }

    // ---- 6. in the tail phase, hand the shallowest pending sibling to the
    //         ring every 32 x `budget` evaluations of the warp, in one
    //         reservation ---------------------------------------------------
    {
      bool trig = false;    // to the ring (the same in every lane)
      bool btrig = false;   // to the block's queue (the same in every lane)
      if (CCD_COLD(tail_phase)) {
        const int ne = __popc(__ballot_sync(FULL, evaluate));
        const long long ws = wc.wsince + ne;
        trig = ws >= 32ll * A.budget;
        __syncwarp(FULL);
        if (lane == 0) {
          wc.n_eval_tail += ne;
          wc.wsince = trig ? 0 : ws;
        }
        // a warp of the block idles and few units wait in the block's queue
        int b = 0;
        if (!trig && lane == 0)
          b = *(volatile int *)&BQ.idle > 0 && vload(&BQ.tail) - vload(&BQ.head) < kBQMax / 4;
        btrig = __shfl_sync(FULL, b, 0) != 0;
      }
      const bool want_exp = (trig || btrig) && have && !unit_end;
      if (CCD_COLD((trig || btrig) && __any_sync(FULL, want_exp))) {   // (trig, btrig are the same in every lane)
        Node S{0, 0, 0, 0, 0, 0};
        int dS = 0;
        if (want_exp) {
          if (deep) {
            dS = shallowest_pending(K, N, depth, root_depth, cut, S);
          } else {
            const int d = shallowest_owed(N, depth - rb, root_depth - rb, pend, axlo, axhi, cut, S);
            dS = d > 0 ? rb + d : 0;
          }
        }
        const unsigned xm = __ballot_sync(FULL, dS > 0);
        if (xm && btrig) {
          // block queue: reserve up to one cell per lane with a sibling
          unsigned long long pos0 = ~0ull;
          int mm = 0;
          if (lane == 0) {
            for (int tries = 0; tries < 32; ++tries) {
              const unsigned long long t = vload(&BQ.tail), h = vload(&BQ.head);
              const unsigned long long room = t - h >= kBQMax ? 0ull : kBQMax - (t - h);
              mm = (int)min((unsigned long long)__popc(xm), room);
              if (mm == 0) break;
              if (atomicCAS(&BQ.tail, t, t + mm) == t) {
                pos0 = t;
                atomicAdd(&BQ.local, mm);   // counted before any of them is visible
                break;
              }
            }
          }
          pos0 = __shfl_sync(FULL, pos0, 0);
          mm = __shfl_sync(FULL, mm, 0);
          const int rank = __popc(xm & lt_mask);
          if (pos0 != ~0ull && dS > 0 && rank < mm) {
            const unsigned long long pos = pos0 + rank;
            const int cell = (int)(pos % kBQ);
            // the cell's previous occupant (kBQ positions back) was taken
            // already; wait until its taker has freed it
            bool freed = true;
            for (int spin = 0; vload(&BQ.seq[cell]) != pos; ++spin) {
              if (spin > (1 << 20)) {
                atomicExch(&ctl->status, CCD_ETIMEOUT);
                freed = false;
                break;
              }
              __nanosleep(32);
            }
            if (freed) {
              if (tq != kInfBits) {
                if (A.mode == 0)
                  atomicMin(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf], tq);
                else if (A.mode == 2)
                  atomicMin(&A.toi_scene[SID[tid]], tq);
                else
                  atomicMin(&ctl->toi_bits, tq);
              }
              atomicAdd(&A.qiters[q], (unsigned long long)cnt);
              cap_left = min(kBudgetWindow, cap_left - cnt);   // (the query's budget is shared from now on)
              cnt = 0;
              whole = false;
              BQ.w[cell][0] = pack1(S.n0, S.l0);
              BQ.w[cell][1] = pack1(S.n1, S.l1);
              BQ.w[cell][2] = pack1(S.n2, S.l2);
              BQ.q[cell] = (uint32_t)q;
              __threadfence_block();
              *(volatile unsigned long long *)&BQ.seq[cell] = pos + 1;
              root_depth = dS;
              atomicAdd(&wc.n_don, 1u);
            }
          }
        } else if (xm) {
          unsigned long long pos0 = ~0ull;
          if (lane == 0) {
            pos0 = ring_reserve(&ctl->q_tail, &ctl->q_head, (unsigned long long)__popc(xm), ring_cap >> 2);
            // count the new units before any of them becomes visible
            if (pos0 != ~0ull) {
              atomicAdd(&ctl->pending, (unsigned long long)__popc(xm));
              __threadfence();
            }
          }
          pos0 = __shfl_sync(FULL, pos0, 0);
          __syncwarp(FULL);
          if (pos0 != ~0ull && dS > 0) {
            // publish what the taker reads before the item becomes visible
            if (tq != kInfBits) {
              if (A.mode == 0)
                atomicMin(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf], tq);
              else if (A.mode == 2)
                atomicMin(&A.toi_scene[SID[tid]], tq);
              else
                atomicMin(&ctl->toi_bits, tq);
            }
            atomicAdd(&A.qiters[q], (unsigned long long)cnt);
            cap_left = min(kBudgetWindow, cap_left - cnt);   // (the query's budget is shared from now on)
            cnt = 0;
            whole = false;
            ring_write(A.ring, A.ring_mask, pos0 + __popc(xm & lt_mask), (uint32_t)q, S, &ctl->status);
            root_depth = dS;
            atomicAdd(&wc.n_exp, 1u);
          }
        }
      }
    }

    // ---- 7. finish the unit ------------------------------------------------
    if (have && unit_end) {
      // (modes 1 and 2 published every accept already: t* and the scene's
      // t*; the global t* of mode 2 and the per-pair result of mode 0 here)
      if (tq != kInfBits && A.mode != 1) {
        if (A.mode == 0)
          atomicMin(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf], tq);
        atomicMin(&ctl->toi_bits, tq);
      }
      if (flags) atomicOr(&A.qflags[q], flags);
      if (!whole && cnt) atomicAdd(&A.qiters[q], (unsigned long long)cnt);
      if (blocal) atomicSub(&BQ.local, 1);
      have = false;
    }
    // units that ended: one pending decrement per warp for 64 of them (the
    // count stays an over-estimate until the warp flushes, at the latest
    // before it idles); units of the block queue are counted in BQ.local
    ended_acc += __popc(__ballot_sync(FULL, unit_end && !blocal));
    if (unit_end) blocal = false;
    if (ended_acc >= 64) {
      if (lane == 0) atomicAdd(&ctl->pending, (unsigned long long)(-(long long)ended_acc));
      ended_acc = 0;
    }
  }

  // A warp also leaves after kIdleRounds idle rounds, so a unit that can
  // never finish (a pending count that does not return to zero) ends the
  // launch instead of holding the GPU; the last warp to leave then records
  // CCD_ETIMEOUT.  (A warp leaves a finished launch only after the count it
  // read was zero, and the count cannot rise again once every query is out.)
  if (lane == 0) {
    __threadfence();   // this warp's updates of the count before its departure
    if (atomicAdd(&ctl->n_left, 1u) == gridDim.x * (blockDim.x >> 5) - 1) {
      __threadfence();   // every other warp's updates before the count is read
      if (ld_relaxed_u64(&ctl->pending) != 0) atomicCAS(&ctl->status, CCD_OK, CCD_ETIMEOUT);
    }
  }
  if (n_eval) atomicAdd(&ctl->n_intervals, (unsigned long long)n_eval);
  __syncwarp(FULL);
  if (lane == 0) {
    if (wc.n_exp) atomicAdd(&ctl->n_exported, (unsigned long long)wc.n_exp);
    if (wc.n_cap) atomicAdd(&ctl->n_capped, (unsigned long long)wc.n_cap);
    if (wc.n_don) atomicAdd(&ctl->n_donated, (unsigned long long)wc.n_don);
    if (wc.n_eval_tail) atomicAdd(&ctl->n_intervals_tail, (unsigned long long)wc.n_eval_tail);
  }
  if (n_eval64) atomicAdd(&ctl->n_intervals_fp64, (unsigned long long)n_eval64);
  if (lane == 0) atomicMax(&ctl->t_end, globaltimer());
}
#undef ST

// The narrow phase on query records (k_prepare_queries), and the same loop
// with each lane setting its queries up itself (no record buffer: the
// allocation-free entry point).  Two kernels, so that neither carries the
// other's code.
__global__ void __launch_bounds__(kNarrowThreads, 3) k_narrow(NarrowArgs A) { narrow_body<true>(A); }
__global__ void __launch_bounds__(kNarrowThreads, 3) k_narrow_setup(NarrowArgs A) { narrow_body<false>(A); }

// One thread per primitive: the per-primitive part of the query set-up
// (records described at kVertWords).
__global__ void k_prepare_prims(NarrowArgs A) {
  if (A.only_if_rerun && A.ctl->rerun == 0) return;
  const int64_t nP = A.nV + A.nE + A.nF;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nP; i += (int64_t)gridDim.x * blockDim.x) {
    if (i < A.nV) {
      double p0[3], p1[3];
      load_pos(A.V0, A.V1, A.nV, (int)i, p0, p1);
      double *r = A.prims + kVertWords * i;
      double e[3];
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        const unsigned long long a = abs_max_bits(p0[x], p1[x]);
        e[x] = eps_of(a > kM0 ? a : kM0);
      }
      store2(r, e[0], e[1]);
      store2(r + 2, e[2], 0.0);
    } else if (i < A.nV + A.nE) {
      const int64_t k = i - A.nV;
      const int a0 = __ldg(&A.E[2 * k]), a1 = __ldg(&A.E[2 * k + 1]);
      double p0[3], p1[3], q0[3], q1[3], c0[3], dc[3], e[3];
      load_pos(A.V0, A.V1, A.nV, a0, p0, p1);
      load_pos(A.V0, A.V1, A.nV, a1, q0, q1);
      vec_of(q0, q1, p0, p1, c0, dc);   // A1 - A0
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        unsigned long long m = kM0;
        unsigned long long t = abs_max_bits(p0[x], p1[x]);
        m = t > m ? t : m;
        t = abs_max_bits(q0[x], q1[x]);
        m = t > m ? t : m;
        e[x] = eps_of(m);
      }
      double *r = A.prims + kVertWords * A.nV + kEdgeWords * k;
      store2(r, c0[0], c0[1]);
      store2(r + 2, c0[2], dc[0]);
      store2(r + 4, dc[1], dc[2]);
      store2(r + 6, e[0], e[1]);
      store2(r + 8, e[2], __longlong_as_double((long long)edge_weight(c0, dc)));
    } else {
      const int64_t k = i - A.nV - A.nE;
      const int t0 = __ldg(&A.F[3 * k]), t1 = __ldg(&A.F[3 * k + 1]), t2 = __ldg(&A.F[3 * k + 2]);
      double p0[3], p1[3], q0[3], q1[3], s0[3], s1[3], c0a[3], dca[3], c0b[3], dcb[3], e[3];
      load_pos(A.V0, A.V1, A.nV, t0, p0, p1);
      load_pos(A.V0, A.V1, A.nV, t1, q0, q1);
      load_pos(A.V0, A.V1, A.nV, t2, s0, s1);
      vec_of(q0, q1, p0, p1, c0a, dca);   // T1 - T0
      vec_of(s0, s1, p0, p1, c0b, dcb);   // T2 - T0
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        unsigned long long m = kM0;
        unsigned long long t = abs_max_bits(p0[x], p1[x]);
        m = t > m ? t : m;
        t = abs_max_bits(q0[x], q1[x]);
        m = t > m ? t : m;
        t = abs_max_bits(s0[x], s1[x]);
        m = t > m ? t : m;
        e[x] = eps_of(m);
      }
      double *r = A.prims + kVertWords * A.nV + kEdgeWords * A.nE + kFaceWords * k;
      store2(r, c0a[0], c0a[1]);
      store2(r + 2, c0a[2], dca[0]);
      store2(r + 4, dca[1], dca[2]);
      store2(r + 6, c0b[0], c0b[1]);
      store2(r + 8, c0b[2], dcb[0]);
      store2(r + 10, dcb[1], dcb[2]);
      store2(r + 12, e[0], e[1]);
      store2(r + 14, e[2], __longlong_as_double((long long)edge_weight(c0a, dca)));
      store2(r + 16, __longlong_as_double((long long)edge_weight(c0b, dcb)), 0.0);
    }
  }
}

// The record of query q from its primitives' records and the two vertices of
// w (the vector P - T0 or A0 - B0; the edge vectors, eps and L_u, L_v come
// from the primitives), written axis by axis so that only one axis's values
// are live at a time: the same operations on the same operands as
// setup_query + setup_tail, so every word is bit-identical.
__device__ __forceinline__ void prepare_record(const NarrowArgs &A, int64_t q, int &first_vertex) {
  const double *__restrict__ P = A.prims;
  const int64_t S = A.rec_stride;
  unsigned long long *__restrict__ rec = A.qrec;
  float *__restrict__ r32 = (float *)(A.qrec + kRecWords * S);
  const double *r1, *r2, *e1, *e2;   // vectors 1, 2 (c0 at [0, 3), dc at [3, 6)) and their eps words
  int xi, yi;                        // w = X - Y
  unsigned long long Lu, Lv;
  const bool vf = q < A.n_vf;
  if (vf) {
    const int v = __ldg(&A.vf[2 * q]), f = __ldg(&A.vf[2 * q + 1]);
    xi = v;
    yi = __ldg(&A.F[3 * (int64_t)f]);
    const double *rf = P + kVertWords * A.nV + kEdgeWords * A.nE + kFaceWords * (int64_t)f;
    r1 = rf;
    r2 = rf + 6;
    e1 = P + kVertWords * (int64_t)v;
    e2 = rf + 12;
    Lu = dbits(__ldg(&rf[15]));
    Lv = dbits(__ldg(&rf[16]));
  } else {
    const int64_t r = q - A.n_vf;
    const int a = __ldg(&A.ee[2 * r]), b = __ldg(&A.ee[2 * r + 1]);
    xi = __ldg(&A.E[2 * (int64_t)a]);
    yi = __ldg(&A.E[2 * (int64_t)b]);
    r1 = P + kVertWords * A.nV + kEdgeWords * (int64_t)a;
    r2 = P + kVertWords * A.nV + kEdgeWords * (int64_t)b;
    e1 = r1 + 6;
    e2 = r2 + 6;
    Lu = dbits(__ldg(&r1[9]));
    Lv = dbits(__ldg(&r2[9]));
  }
  first_vertex = xi;
  const bool no_sep = A.min_sep == 0.0;   // (one FP64 comparison per query, not per axis)
  unsigned long long Lt = 0;
#pragma unroll 1
  for (int x = 0; x < 3; ++x) {
    const double X0 = __ldg(&A.V0[x * A.nV + xi]), X1 = __ldg(&A.V1[x * A.nV + xi]);
    const double Y0 = __ldg(&A.V0[x * A.nV + yi]), Y1 = __ldg(&A.V1[x * A.nV + yi]);
    double c0[3], dc[3];
    c0[0] = __dsub_rn(X0, Y0);
    dc[0] = __dsub_rn(__dsub_rn(X1, Y1), c0[0]);
    c0[1] = __ldg(&r1[x]);
    dc[1] = __ldg(&r1[3 + x]);
    c0[2] = __ldg(&r2[x]);
    dc[2] = __ldg(&r2[3 + x]);
    AxisSetup o;
    setup_axis(o, c0, dc, dmax_pos(__ldg(&e1[x]), __ldg(&e2[x])), A.min_sep, no_sep, A.delta);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      rec[(3 * j + x) * S + q] = dbits(c0[j]);
      rec[(9 + 3 * j + x) * S + q] = dbits(dc[j]);
      r32[(2 * (3 * j + x)) * S + q] = o.c0f[j];
      r32[(2 * (3 * j + x) + 1) * S + q] = o.dcf[j];
    }
    rec[(18 + x) * S + q] = dbits(o.e);   // (e > 0: its ordered key is its bits)
    r32[(18 + 5 * x) * S + q] = o.tn;
    r32[(19 + 5 * x) * S + q] = o.tm;
    r32[(20 + 5 * x) * S + q] = o.wn;
    r32[(21 + 5 * x) * S + q] = o.cc0;
    r32[(22 + 5 * x) * S + q] = o.cdc;
    Lt = o.st > Lt ? o.st : Lt;
  }
  rec[21 * S + q] = (Lt < kKeyFloor ? 0ull : Lt) | (vf ? (1ull << 63) : 0ull);
  rec[22 * S + q] = Lu < kKeyFloor ? 0ull : Lu;
  rec[23 * S + q] = Lv < kKeyFloor ? 0ull : Lv;
}

// One thread per query: the query's set-up from its primitives' records
// (k_prepare_prims) and two vertices, stored as a record, so that the narrow
// kernel's lanes set up a unit from coalesced loads with no FP64 work.
__global__ void k_prepare_queries(NarrowArgs A) {
  if (A.only_if_rerun && A.ctl->rerun == 0) return;
  if (A.counts_from_ctl) {
    A.n_vf = A.ctl->pair_counts[0];
    A.n_ee = A.ctl->pair_counts[1];
    if (A.ee_end > 0) A.ee = A.vf + 2 * (A.ee_end - A.n_ee);
  }
  const int64_t nq = A.n_vf + A.n_ee;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
    int v0;
    prepare_record(A, q, v0);
    if (A.n_scenes > 0) A.qsid[q] = scene_of(A.voff, A.n_scenes, v0);
  }
}

// Zero-TOI rule (appendix "Zero time of impact and minimum separation"): when
// the first pass found t* = 0, reset the narrow-phase state for a second
// pass (min_sep = 0, intervals at t = 0 always split) ...
__global__ void k_nozero_prepare(DevCtl *ctl) {
  ctl->rerun = ctl->toi_bits == 0 ? 1 : 0;
  if (ctl->rerun) {
    ctl->q_next = 0;
    ctl->pending = 0;
    ctl->toi_bits = kInfBits;
    ctl->t_start = ctl->t_exhausted = ctl->t_end = 0;
    ctl->n_left = 0;
  }
}

// ... and scale its result by 0.8.
__global__ void k_nozero_finish(DevCtl *ctl) {
  if (ctl->rerun && ctl->toi_bits != kInfBits)
    ctl->toi_bits = dbits(__dmul_rn(0.8, __longlong_as_double((long long)ctl->toi_bits)));
}

__global__ void k_ring_init(RingCell *ring, unsigned long long cap, unsigned long long base) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < cap;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    // the cell that position p (base <= p < base + cap) maps to expects seq == p
    unsigned long long p = base + ((i - (base & (cap - 1))) & (cap - 1));
    ring[i].seq = p;
  }
}

__global__ void k_fill_u64(unsigned long long *p, int64_t n, unsigned long long v) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

__global__ void k_flags_out(const uint32_t *qflags, int64_t n_vf, int64_t n_ee, uint8_t *flags_vf,
                            uint8_t *flags_ee, DevCtl *ctl) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n_vf + n_ee;
       i += (int64_t)gridDim.x * blockDim.x) {
    uint8_t f = (uint8_t)qflags[i];
    if (i < n_vf) {
      if (flags_vf) flags_vf[i] = f;
    } else if (flags_ee) {
      flags_ee[i - n_vf] = f;
    }
  }
  (void)ctl;
}

}  // namespace ccd
