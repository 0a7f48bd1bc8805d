// Narrow phase: conservative interval bisection over (t, u, v) in FP64
// (Section "Narrow-Phase", Algorithm 3, ProcessInterval).
//
// GB300 design
//   * One persistent launch.  Every lane owns a unit of work (a whole query,
//     or a subtree of one) and walks it depth first, left half first.  The
//     split axis depends only on the interval's levels (see split_axis), so
//     every node at a given depth has the same levels and the DFS needs no
//     stack: the path is the binary expansion of the three numerators.
//   * Load balance at interval granularity: after `budget` intervals a lane
//     hands its live intervals (the current one and the pending right
//     siblings) to a device-wide bounded MPMC ring and takes new work; idle
//     lanes drain the ring before fetching new queries.  A single
//     near-degenerate query (tens of thousands of intervals) is thus spread
//     over many lanes, which is the point of the paper's per-interval
//     parallelism, without its level-synchronous launches.
//   * FP64 is the scarce unit on this GPU.  Per interval: 18 DFMA for the two
//     time ends (w, e1, e2 per axis), 24 DFMA for the corner hull and 3 DADD
//     for the width test.  The hull needs only 2 of the 4 (u, v) corners per
//     time end and axis: rounding is monotone, so the minimum of the computed
//     corners is the corner picked by the signs of the computed edge vectors,
//     bit for bit the same as the minimum over all corners.  Comparisons,
//     min/max, dyadic endpoints and the split rule run on the integer pipes.
//   * Earliest-TOI mode: one shared t* (ordered FP64 bits, atomicMin) prunes
//     every query; per-pair mode keeps t* per query.  Either way the result
//     for a query that hits no cap is independent of the traversal order: a
//     pruned interval starts at or after a t* that is already >= the final t*.
//
// Every wait is bounded; on expiry the kernel records CCD_ETIMEOUT and returns.

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
};

__device__ __forceinline__ unsigned long long dbits(double d) {
  return (unsigned long long)__double_as_longlong(d);
}

// Per-query set-up; the reading of the error box and split weights matches the
// oracle's setup_query.  ids: VF (P, T0, T1, T2), EE (A0, A1, B0, B1).
__device__ void setup_query(QueryData &Q, bool vf, const int ids[4], const double *__restrict__ V0,
                            const double *__restrict__ V1, int64_t nV, double min_sep) {
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
  unsigned long long Lt = 0, Lu = 0, Lv = 0;
#pragma unroll
  for (int x = 0; x < 3; ++x) {
    unsigned long long m = 0x03F0000000000000ull;  // 2^-960
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      unsigned long long a = dbits(x0[k][x]) & 0x7FFFFFFFFFFFFFFFull;
      unsigned long long b = dbits(x1[k][x]) & 0x7FFFFFFFFFFFFFFFull;
      m = a > m ? a : m;
      m = b > m ? b : m;
    }
    double eps = __dmul_rn(__longlong_as_double((long long)m), 0x1.8p-48);  // 48 * 2^-53
    double e = __dadd_rn(eps, min_sep);
    e = __longlong_as_double(__double_as_longlong(e) + 1);                   // one ulp up
    Q.ebox_p[x] = f64_ord(e);
    Q.ebox_n[x] = f64_ord(-e);
    double st = __dadd_rn(dabs_int(Q.dc[0][x]), dabs_int(Q.dc[1][x]));
    st = __dadd_rn(st, dabs_int(Q.dc[2][x]));
    unsigned long long sb = dbits(st);
    Lt = sb > Lt ? sb : Lt;
    unsigned long long u0 = dbits(dabs_int(Q.c0[1][x]));
    unsigned long long u1 = dbits(dabs_int(__dadd_rn(Q.c0[1][x], Q.dc[1][x])));
    unsigned long long v0 = dbits(dabs_int(Q.c0[2][x]));
    unsigned long long v1 = dbits(dabs_int(__dadd_rn(Q.c0[2][x], Q.dc[2][x])));
    u0 = u1 > u0 ? u1 : u0;
    v0 = v1 > v0 ? v1 : v0;
    Lu = u0 > Lu ? u0 : Lu;
    Lv = v0 > Lv ? v0 : Lv;
  }
  const unsigned long long kFloor = 0x0DF0000000000000ull;  // 2^-800
  Q.K[0] = Lt < kFloor ? 0 : Lt;
  Q.K[1] = Lu < kFloor ? 0 : Lu;
  Q.K[2] = Lv < kFloor ? 0 : Lv;
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

// ---- bounded MPMC ring of exported intervals -------------------------------
// Cell: sequence number + interval.  Sequence protocol: a cell at position p
// is free for a writer when seq == p, holds data when seq == p + 1, and is
// released for the next lap (seq = p + cap) after it has been read.

__device__ __forceinline__ unsigned long long pack1(uint64_t n, int l) {
  return n | ((unsigned long long)l << 54);
}

__device__ bool ring_push(RingCell *ring, unsigned long long mask, unsigned long long *tail, uint32_t q,
                          const Node &N, int *status) {
  unsigned long long pos = ld_relaxed_u64(tail);
  for (int spin = 0; spin < (1 << 20); ++spin) {
    RingCell *c = &ring[pos & mask];
    unsigned long long seq = ld_acquire_u64(&c->seq);
    long long dif = (long long)(seq - pos);
    if (dif == 0) {
      if (atomicCAS(tail, pos, pos + 1) == pos) {
        c->w[0] = pack1(N.n0, N.l0);
        c->w[1] = pack1(N.n1, N.l1);
        c->w[2] = pack1(N.n2, N.l2);
        c->q = q;
        st_release_u64(&c->seq, pos + 1);
        return true;
      }
      pos = ld_relaxed_u64(tail);
    } else if (dif < 0) {
      __nanosleep(64);  // full: readers are draining it
      pos = ld_relaxed_u64(tail);
    } else {
      pos = ld_relaxed_u64(tail);
    }
  }
  atomicExch(status, CCD_ETIMEOUT);
  return false;
}

__device__ bool ring_pop(RingCell *ring, unsigned long long mask, unsigned long long *head, uint32_t &q,
                         Node &N) {
  unsigned long long pos = ld_relaxed_u64(head);
  for (int spin = 0; spin < 64; ++spin) {
    RingCell *c = &ring[pos & mask];
    unsigned long long seq = ld_acquire_u64(&c->seq);
    long long dif = (long long)(seq - (pos + 1));
    if (dif == 0) {
      if (atomicCAS(head, pos, pos + 1) == pos) {
        const unsigned long long w0 = c->w[0], w1 = c->w[1], w2 = c->w[2];
        const unsigned long long m54 = (1ull << 54) - 1;
        q = c->q;
        N.n0 = w0 & m54;
        N.n1 = w1 & m54;
        N.n2 = w2 & m54;
        N.l0 = (int)(w0 >> 54);
        N.l1 = (int)(w1 >> 54);
        N.l2 = (int)(w2 >> 54);
        st_release_u64(&c->seq, pos + mask + 1);
        return true;
      }
      pos = ld_relaxed_u64(head);
    } else if (dif < 0) {
      return false;  // empty
    } else {
      pos = ld_relaxed_u64(head);
    }
  }
  return false;
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

}  // namespace

constexpr int kIdleSpinLimit = 1 << 16;   // ~0.05 s of 512 ns naps, then a lane retires

__global__ void __launch_bounds__(kNarrowThreads, 3)
k_narrow(NarrowArgs A) {
  DevCtl *ctl = A.ctl;
  if (A.counts_from_ctl) {
    A.n_vf = ctl->pair_counts[0];
    A.n_ee = ctl->pair_counts[1];
  }
  const int64_t nq = A.n_vf + A.n_ee;
  const int lane = threadIdx.x & 31;
  const unsigned long long delta_bits = dbits(A.delta);
  const unsigned long long ring_cap = A.ring_mask + 1;

  QueryData Q;
  bool vf = false;
  bool have = false, fresh = false, whole = false, exhausted = false;
  int64_t q = 0;
  Node N{0, 0, 0, 0, 0, 0};
  int depth = 0, root_depth = 0;
  unsigned long long tq = kInfBits;          // bits of this unit's best t*
  long long cnt = 0, cap_left = 0;
  unsigned flags = 0;
  long long n_eval = 0, n_exp = 0, n_cap = 0;
  int idle_spins = 0;

  while (true) {
    // ---- 1. acquire work: exported intervals first, then new queries ------
    if (!have && ld_relaxed_u64(&ctl->q_head) != ld_relaxed_u64(&ctl->q_tail)) {
      uint32_t qq;
      if (ring_pop(A.ring, A.ring_mask, &ctl->q_head, qq, N)) {
        q = qq;
        have = fresh = true;
        whole = false;
      }
    }
    if (!have && !exhausted) {
      unsigned m = __activemask();
      int leader = __ffs(m) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(&ctl->q_next, (unsigned long long)__popc(m));
      base = __shfl_sync(m, base, leader);
      unsigned long long mine = base + __popc(m & ((1u << lane) - 1u));
      bool got = (int64_t)mine < nq;
      if (got) {
        q = (int64_t)mine;
        have = fresh = whole = true;
        N = Node{0, 0, 0, 0, 0, 0};
      } else {
        exhausted = true;
      }
      unsigned gm = __ballot_sync(m, got);
      if (lane == leader && gm) atomicAdd(&ctl->pending, (unsigned long long)__popc(gm));
      __syncwarp(m);
    }
    if (!have) {
      if (ld_relaxed_u64(&ctl->q_head) == ld_relaxed_u64(&ctl->q_tail)) {
        if (ld_relaxed_u64(&ctl->pending) == 0 || ++idle_spins > kIdleSpinLimit) break;
        __nanosleep(512);
      }
      continue;
    }
    idle_spins = 0;

    // ---- 2. set up a new unit ---------------------------------------------
    if (fresh) {
      int ids[4];
      query_ids(q, A.n_vf, A.vf, A.ee, A.E, A.F, ids, vf);
      setup_query(Q, vf, ids, A.V0, A.V1, A.nV, A.min_sep);
      depth = root_depth = N.depth();
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
        cap_left = A.max_iter - (long long)ld_relaxed_u64(&A.qiters[q]);
      }
      fresh = false;
    }

    // ---- 3. ProcessInterval on the current node ---------------------------
    unsigned long long cut = tq;
    if (A.mode == 1) {
      unsigned long long g = ld_relaxed_u64(&ctl->toi_bits);
      cut = g < cut ? g : cut;
    }
    const double tl = dyadic(N.n0, N.l0);
    bool node_done = true;     // false when the node was split (go to its left child)
    bool unit_end = false;
    if (dbits(tl) >= cut) {
      // pruned: starts at or after the current t*
    } else if (vf && dbits(dyadic(N.n1, N.l1)) > dbits(dyadic((1ull << N.l2) - N.n2, N.l2))) {
      // vertex-face: u_lo > 1 - v_lo, the interval lies outside the simplex
    } else if (++cnt > cap_left) {
      // iteration cap: t* = min(t*, earliest left end among the live intervals)
      unsigned long long m = dbits(tl);
      Node W = N;
      for (int d = depth; d > root_depth; --d) {
        int a = last_axis(Q.K, W);
        if ((W.n(a) & 1) == 0) {
          unsigned long long sb = dbits(a == 0 ? dyadic(W.n0 + 1, W.l0) : dyadic(W.n0, W.l0));
          m = sb < m ? sb : m;
        }
        W.up(a);
      }
      tq = m < tq ? m : tq;
      flags |= CCD_FLAG_ITER_CAP;
      ++n_cap;
      --cnt;
      unit_end = true;
    } else {
      ++n_eval;
      const double tr = dyadic(N.n0 + 1, N.l0);
      const double ul = dyadic(N.n1, N.l1), ur = dyadic(N.n1 + 1, N.l1);
      const double vl = dyadic(N.n2, N.l2), vr = dyadic(N.n2 + 1, N.l2);
      Box3 B;
      inclusion(Q, vf, tl, tr, ul, ur, vl, vr, B);
      bool miss = false, inside = true, narrow = true;
#pragma unroll
      for (int x = 0; x < 3; ++x) {
        long long lo = f64_ord(B.lo[x]), hi = f64_ord(B.hi[x]);
        miss |= (lo > Q.ebox_p[x]) | (hi < Q.ebox_n[x]);
        inside &= (lo >= Q.ebox_n[x]) & (hi <= Q.ebox_p[x]);
        narrow &= dbits(__dsub_rn(B.hi[x], B.lo[x])) < delta_bits;
      }
      if (!miss) {
        bool accept = narrow || inside;
        int a = -1;
        if (!accept) {
          a = split_axis(Q.K, N);
          if (a < 0) {
            accept = true;
            flags |= CCD_FLAG_LEVEL_CAP;
          }
        }
        if (accept) {
          tq = dbits(tl);
          if (A.mode == 1) atomicMin(&ctl->toi_bits, tq);
        } else {
          N.down_left(a);
          depth += 1;
          node_done = false;
        }
      }
    }

    // ---- 4. next node: backtrack to the deepest pending right sibling ------
    if (node_done && !unit_end) {
      while (true) {
        if (depth == root_depth) {
          unit_end = true;
          break;
        }
        int a = last_axis(Q.K, N);
        if ((N.n(a) & 1) == 0) {
          N.add(a, 1);
          break;
        }
        N.up(a);
        depth -= 1;
      }
    }

    // ---- 5. hand out the live intervals after `budget` evaluations --------
    if (!unit_end && cnt >= A.budget) {
      unsigned long long head = ld_relaxed_u64(&ctl->q_head);
      unsigned long long tail = ld_relaxed_u64(&ctl->q_tail);
      if (tail - head < (ring_cap >> 2)) {
        int nexp = 1;
        {
          Node W = N;
          for (int d = depth; d > root_depth; --d) {
            int a = last_axis(Q.K, W);
            nexp += (W.n(a) & 1) == 0;
            W.up(a);
          }
        }
        // publish what the takers read before they can pop the items
        if (tq != kInfBits) {
          if (A.mode == 0)
            atomicMin(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf], tq);
          else
            atomicMin(&ctl->toi_bits, tq);
        }
        atomicAdd(&A.qiters[q], (unsigned long long)cnt);
        atomicAdd(&ctl->pending, (unsigned long long)nexp);
        bool ok = ring_push(A.ring, A.ring_mask, &ctl->q_tail, (uint32_t)q, N, &ctl->status);
        Node W = N;
        for (int d = depth; d > root_depth && ok; --d) {
          int a = last_axis(Q.K, W);
          if ((W.n(a) & 1) == 0) {
            Node S = W;
            S.add(a, 1);
            ok = ring_push(A.ring, A.ring_mask, &ctl->q_tail, (uint32_t)q, S, &ctl->status);
          }
          W.up(a);
        }
        unsigned long long occ = ld_relaxed_u64(&ctl->q_tail) - ld_relaxed_u64(&ctl->q_head);
        if (occ > ld_relaxed_u64(&ctl->queue_peak)) atomicMax(&ctl->queue_peak, occ);
        n_exp += nexp;
        unit_end = true;
        cnt = 0;   // already added to qiters
      }
    }

    // ---- 6. finish the unit ------------------------------------------------
    if (unit_end) {
      if (tq != kInfBits) {
        if (A.mode == 0)
          atomicMin(q < A.n_vf ? &A.toi_vf_bits[q] : &A.toi_ee_bits[q - A.n_vf], tq);
        atomicMin(&ctl->toi_bits, tq);
      }
      if (flags) atomicOr(&A.qflags[q], flags);
      if (!whole && cnt) atomicAdd(&A.qiters[q], (unsigned long long)cnt);
      atomicAdd(&ctl->pending, ~0ull);   // -1
      have = false;
    }
  }

  if (n_eval) atomicAdd(&ctl->n_intervals, (unsigned long long)n_eval);
  if (n_exp) atomicAdd(&ctl->n_exported, (unsigned long long)n_exp);
  if (n_cap) atomicAdd(&ctl->n_capped, (unsigned long long)n_cap);
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
