// Serving runtime: continuous batching of CCD steps that arrive one scene at a
// time (include/ccd.h, "Serving").
//
// Clients write each scene straight into a pinned host arena (ccd_server_request
// hands out the space, ccd_server_submit queues it).  A scheduler thread forms
// a batch from the queued scenes whenever one of its slots is free, bounded by
// scene count, box count and the slot's share of the memory cap, and runs it
// on the slot's own stream and context: one host-to-device copy of the batch's
// contiguous arena range, one kernel that unpacks the scenes into the batched
// layout (structure of arrays, global vertex ids, offsets), ccd_step_batch,
// and one device-to-host copy of the per-scene results.  Slots overlap: one
// batch copies while another computes.  A host callback on the stream marks
// the batch's scenes done; the arena space is recycled in arrival order.

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

inline int64_t align_up(int64_t x, int64_t a) { return (x + a - 1) / a * a; }

// Layout of one scene in the arena: V0 [3][nV], V1 [3][nV] (doubles), E
// [nE][2], F [nF][3] (int32, vertex ids local to the scene), 256-byte aligned.
struct Block {
  int64_t off, bytes;
  int64_t nV, nE, nF;
  int64_t oV1, oE, oF;   // byte offsets within the block
};

Block make_block(int64_t off, int64_t nV, int64_t nE, int64_t nF) {
  Block b;
  b.off = off;
  b.nV = nV;
  b.nE = nE;
  b.nF = nF;
  b.oV1 = align_up(3 * nV * 8, 256);
  b.oE = b.oV1 + align_up(3 * nV * 8, 256);
  b.oF = b.oE + align_up(2 * nE * 4, 256);
  b.bytes = b.oF + align_up(3 * nF * 4, 256);
  if (b.bytes == 0) b.bytes = 256;
  return b;
}

// Per-scene descriptor of a batch (device copy read by k_unpack).
struct Desc {
  int64_t src;                 // byte offset of the scene's block in the batch's staging copy
  int64_t nV, nE, nF;
  int64_t voff, eoff, foff;    // offsets of the scene in the batched arrays
  int64_t oV1, oE, oF;
};

// One CTA per scene: copy its coordinates into the batched structure of
// arrays and its edges and faces with vertex ids made global.
__global__ void k_unpack(const unsigned char *__restrict__ staging, const Desc *__restrict__ D, int n,
                         int64_t nV_all, double *V0, double *V1, int32_t *E, int32_t *F, int64_t *voff,
                         int64_t *eoff, int64_t *foff) {
  const int s = blockIdx.x;
  if (s >= n) return;
  const Desc d = D[s];
  const double *v0 = (const double *)(staging + d.src);
  const double *v1 = (const double *)(staging + d.src + d.oV1);
  const int32_t *e = (const int32_t *)(staging + d.src + d.oE);
  const int32_t *f = (const int32_t *)(staging + d.src + d.oF);
  for (int64_t i = threadIdx.x; i < 3 * d.nV; i += blockDim.x) {
    const int64_t a = i / d.nV, k = i - a * d.nV;
    V0[a * nV_all + d.voff + k] = v0[i];
    V1[a * nV_all + d.voff + k] = v1[i];
  }
  const int vo = (int)d.voff;
  for (int64_t i = threadIdx.x; i < 2 * d.nE; i += blockDim.x) E[2 * d.eoff + i] = e[i] + vo;
  for (int64_t i = threadIdx.x; i < 3 * d.nF; i += blockDim.x) F[3 * d.foff + i] = f[i] + vo;
  if (threadIdx.x == 0) {
    voff[s] = d.voff;
    eoff[s] = d.eoff;
    foff[s] = d.foff;
    if (s == n - 1) {
      voff[n] = d.voff + d.nV;
      eoff[n] = d.eoff + d.nE;
      foff[n] = d.foff + d.nF;
    }
  }
}

struct Request {
  uint64_t id = 0;
  Block blk{};
  bool submitted = false, done = false;
  double t_submit = 0, t_done = 0;
  double toi = 0;
  int status = CCD_OK;
};

struct Slot;

struct Batch {
  std::vector<Request *> reqs;
  int64_t arena_end = 0;       // arena position after the batch's last block
  int64_t bytes = 0;           // device-memory need by the memory model
  std::atomic<bool> done{false};   // set by the stream callback (or a failed launch)
  bool delivered = false;      // results handed to the scenes, slot released
  Slot *slot = nullptr;
  ccd_server *server = nullptr;
};

template <class T>
int grow_dev(T **p, int64_t *cap, int64_t n) {
  if (n <= *cap) return CCD_OK;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t c = std::max<int64_t>(n + n / 4, 1024);
  if (cudaMalloc(p, c * sizeof(T)) != cudaSuccess) return CCD_ENOMEM;
  *cap = c;
  return CCD_OK;
}

template <class T>
int grow_host(T **p, int64_t *cap, int64_t n) {
  if (n <= *cap) return CCD_OK;
  if (*p) cudaFreeHost(*p);
  *p = nullptr;
  *cap = 0;
  const int64_t c = std::max<int64_t>(n + n / 4, 1024);
  if (cudaHostAlloc(p, c * sizeof(T), cudaHostAllocDefault) != cudaSuccess) return CCD_ENOMEM;
  *cap = c;
  return CCD_OK;
}

struct Slot {
  ccd_ctx *ctx = nullptr;
  cudaStream_t stream = nullptr;
  bool busy = false;
  // device buffers
  unsigned char *staging = nullptr;
  int64_t cap_staging = 0;
  double *V0 = nullptr, *V1 = nullptr, *toi = nullptr;
  int64_t cap_V = 0, cap_V1 = 0, cap_toi = 0;
  int32_t *E = nullptr, *F = nullptr;
  int64_t cap_E = 0, cap_F = 0;
  int64_t *offs = nullptr;
  int64_t cap_offs = 0;
  Desc *desc = nullptr;
  int64_t cap_desc = 0;
  // pinned host buffers
  Desc *h_desc = nullptr;
  int64_t cap_h_desc = 0;
  double *h_toi = nullptr;
  int64_t cap_h_toi = 0;
  int32_t *h_status = nullptr;
  int64_t cap_h_status = 0;
  Batch *batch = nullptr;
  bool tuned = false;
};

}  // namespace

struct ccd_server {
  ccd_server_opts opts{};
  int device = 0;
  int64_t slot_mem = 0;        // memory share of one slot
  ccd_memory_model mm{};
  // arena: a ring of pinned bytes; [tail, head) is in use, in arrival order
  unsigned char *arena = nullptr;
  int64_t arena_bytes = 0, head = 0, tail = 0;   // monotonic byte positions
  std::mutex mu;
  std::condition_variable cv_sched, cv_done, cv_space;
  std::deque<Request *> queue;                   // in arrival (= arena) order
  std::unordered_map<uint64_t, Request *> reqs;
  std::deque<Batch *> inflight;                  // in arena order
  int64_t inflight_bytes = 0;                    // memory-model need of the batches on slots
  std::vector<Slot> slots;
  std::thread sched;
  bool stop = false;
  uint64_t next_id = 1;
  ccd_server_stats st{};
  int error = CCD_OK;
};

namespace {

int64_t est_bytes(const ccd_server *S, int64_t boxes, int64_t scenes) {
  const int64_t pairs = std::max<int64_t>(1 << 20, S->opts.pairs_per_box > 0 ? (int64_t)(S->opts.pairs_per_box * boxes)
                                                                              : 4 * boxes);
  return S->mm.bytes_fixed + std::max<int64_t>(boxes, 1024) * S->mm.bytes_per_box + scenes * S->mm.bytes_per_scene +
         pairs * S->mm.bytes_per_pair;
}

void CUDART_CB on_batch_done(void *arg);

// Under S->mu: hand the results of finished batches to their scenes, release
// their slots, and recycle arena space in arrival order.
void finish_batches(ccd_server *S) {
  const double t = now_s();
  bool any = false;
  for (Batch *b : S->inflight) {
    if (b->delivered || !b->done.load(std::memory_order_acquire)) continue;
    Slot *sl = b->slot;
    const int status = sl->h_status[0];
    for (size_t i = 0; i < b->reqs.size(); ++i) {
      Request *r = b->reqs[i];
      r->toi = sl->h_toi[i];
      r->status = status;
      r->t_done = t;
      r->done = true;
      S->st.n_done += 1;
      S->st.sum_latency_ms += (t - r->t_submit) * 1e3;
    }
    sl->busy = false;
    sl->batch = nullptr;
    b->delivered = true;
    S->inflight_bytes -= b->bytes;
    any = true;
  }
  while (!S->inflight.empty() && S->inflight.front()->delivered) {
    Batch *b = S->inflight.front();
    S->tail = b->arena_end;
    S->inflight.pop_front();
    delete b;
  }
  if (any) {
    S->cv_done.notify_all();
    S->cv_space.notify_all();
  }
}

int run_batch(ccd_server *S, Slot &sl, Batch *b) {
  const int n = (int)b->reqs.size();
  int64_t nV = 0, nE = 0, nF = 0;
  const int64_t first = b->reqs.front()->blk.off;
  int64_t last_end = first;
  for (Request *r : b->reqs) {
    nV += r->blk.nV;
    nE += r->blk.nE;
    nF += r->blk.nF;
    last_end = r->blk.off + r->blk.bytes;
  }
  const int64_t span = last_end - first;   // blocks never wrap: a contiguous range
  int rc = CCD_OK;
  if ((rc = grow_dev(&sl.staging, &sl.cap_staging, span)) || (rc = grow_dev(&sl.V0, &sl.cap_V, 3 * nV)) ||
      (rc = grow_dev(&sl.V1, &sl.cap_V1, 3 * nV)) || (rc = grow_dev(&sl.E, &sl.cap_E, 2 * nE)) ||
      (rc = grow_dev(&sl.F, &sl.cap_F, 3 * nF)) || (rc = grow_dev(&sl.offs, &sl.cap_offs, 3 * (int64_t)(n + 1))) ||
      (rc = grow_dev(&sl.toi, &sl.cap_toi, n)) || (rc = grow_dev(&sl.desc, &sl.cap_desc, n)) ||
      (rc = grow_host(&sl.h_desc, &sl.cap_h_desc, n)) || (rc = grow_host(&sl.h_toi, &sl.cap_h_toi, n)) ||
      (rc = grow_host(&sl.h_status, &sl.cap_h_status, 1)))
    return rc;
  int64_t vo = 0, eo = 0, fo = 0;
  for (int i = 0; i < n; ++i) {
    const Block &k = b->reqs[i]->blk;
    Desc &d = sl.h_desc[i];
    d.src = k.off - first;
    d.nV = k.nV;
    d.nE = k.nE;
    d.nF = k.nF;
    d.voff = vo;
    d.eoff = eo;
    d.foff = fo;
    d.oV1 = k.oV1;
    d.oE = k.oE;
    d.oF = k.oF;
    vo += k.nV;
    eo += k.nE;
    fo += k.nF;
  }
  const int64_t apos = first % S->arena_bytes;
  b->server = S;
  cudaStream_t s = sl.stream;
  if (cudaMemcpyAsync(sl.staging, S->arena + apos, span, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(sl.desc, sl.h_desc, n * sizeof(Desc), cudaMemcpyHostToDevice, s) != cudaSuccess)
    return CCD_ECUDA;
  int64_t *voff = sl.offs, *eoff = sl.offs + (n + 1), *foff = sl.offs + 2 * (n + 1);
  k_unpack<<<n, 256, 0, s>>>(sl.staging, sl.desc, n, nV, sl.V0, sl.V1, sl.E, sl.F, voff, eoff, foff);
  if (cudaGetLastError() != cudaSuccess) return CCD_ECUDA;
  if (S->opts.autotune && !sl.tuned) {
    // tune the slot's context on its first batch (synchronous)
    ccd_tuning t;
    rc = ccd_autotune_batch(sl.ctx, n, voff, eoff, foff, sl.V0, sl.V1, nV, sl.E, nE, sl.F, nF, 2, &t, s);
    if (rc) return rc;
    sl.tuned = true;
  }
  rc = ccd_step_batch(sl.ctx, n, voff, eoff, foff, sl.V0, sl.V1, nV, sl.E, nE, sl.F, nF, S->opts.delta,
                      S->opts.min_sep, S->opts.max_iter, sl.toi, s);
  if (rc) return rc;
  if ((rc = ccd_status_async(sl.ctx, sl.h_status, s))) return rc;
  if (cudaMemcpyAsync(sl.h_toi, sl.toi, n * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CCD_ECUDA;
  if (cudaLaunchHostFunc(s, on_batch_done, b) != cudaSuccess) return CCD_ECUDA;
  return CCD_OK;
}

void scheduler(ccd_server *S) {
  cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    finish_batches(S);
    Slot *free_slot = nullptr;
    for (Slot &sl : S->slots)
      if (!sl.busy) {
        free_slot = &sl;
        break;
      }
    const bool ready = !S->queue.empty() && S->queue.front()->submitted;
    if (S->stop) {
      // scenes handed out but never submitted are dropped
      while (!S->queue.empty() && !S->queue.front()->submitted) S->queue.pop_front();
      if (S->queue.empty() && S->inflight.empty()) break;
    }
    if (!free_slot || !ready) {
      // completions arrive through host callbacks that only set a flag: poll
      S->cv_sched.wait_for(lk, std::chrono::microseconds(50));
      continue;
    }
    // form a batch: queued scenes in arrival order within the slot's limits
    Batch *b = new Batch();
    int64_t boxes = 0;
    while (!S->queue.empty() && S->queue.front()->submitted &&
           (int)b->reqs.size() < S->opts.max_scenes) {
      Request *r = S->queue.front();
      const int64_t nb = r->blk.nV + r->blk.nE + r->blk.nF;
      if (!b->reqs.empty() && (boxes + nb > S->opts.max_boxes ||
                               est_bytes(S, boxes + nb, (int64_t)b->reqs.size() + 1) > S->slot_mem))
        break;
      // blocks of one batch must be contiguous in the arena: stop at a wrap
      if (!b->reqs.empty() && r->blk.off != b->reqs.back()->blk.off + b->reqs.back()->blk.bytes) break;
      b->reqs.push_back(r);
      boxes += nb;
      S->queue.pop_front();
    }
    b->arena_end = b->reqs.back()->blk.off + b->reqs.back()->blk.bytes;
    // admission by memory: each slot holds at most its share of the cap, so
    // the batches in flight together stay within memory_cap
    b->bytes = est_bytes(S, boxes, (int64_t)b->reqs.size());
    S->inflight_bytes += b->bytes;
    S->st.max_batch_bytes = std::max<int64_t>(S->st.max_batch_bytes, b->bytes);
    S->st.max_inflight_bytes = std::max<int64_t>(S->st.max_inflight_bytes, S->inflight_bytes);
    b->slot = free_slot;
    free_slot->busy = true;
    free_slot->batch = b;
    S->inflight.push_back(b);
    S->st.n_batches += 1;
    S->st.max_batch_scenes = std::max<int64_t>(S->st.max_batch_scenes, (int64_t)b->reqs.size());
    lk.unlock();
    const int rc = run_batch(S, *free_slot, b);
    lk.lock();
    if (rc) {
      // the batch could not be launched (nothing of it is in flight on the
      // stream once run_batch returned early): its scenes fail with the status
      cudaStreamSynchronize(free_slot->stream);
      for (Request *r : b->reqs) {
        r->status = rc;
        r->toi = 0;
        r->t_done = now_s();
        r->done = true;
      }
      b->delivered = true;
      b->done.store(true);
      S->inflight_bytes -= b->bytes;
      free_slot->busy = false;
      free_slot->batch = nullptr;
      S->error = rc;
      S->cv_done.notify_all();
    }
  }
}

void CUDART_CB on_batch_done(void *arg) {
  // runs on a CUDA runtime thread: host memory and notifications only
  Batch *b = (Batch *)arg;
  b->done.store(true, std::memory_order_release);
  b->server->cv_sched.notify_all();
  b->server->cv_done.notify_all();
}

}  // namespace

extern "C" {

void ccd_server_default_opts(ccd_server_opts *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->n_slots = 2;
  o->max_scenes = 256;
  o->max_boxes = 1 << 24;
  o->memory_cap = 64ll << 30;
  o->arena_bytes = 1ll << 30;
  o->delta = 1e-6;
  o->min_sep = 0.0;
  o->max_iter = 1000000;
  o->pairs_per_box = 0.0;
}

int ccd_server_create(ccd_server **out, const ccd_server_opts *o, int device) {
  if (!out) return CCD_EINVAL;
  *out = nullptr;
  ccd_server_opts opts;
  ccd_server_default_opts(&opts);
  if (o) opts = *o;
  if (opts.n_slots < 1 || opts.n_slots > 16 || opts.max_scenes < 1 || opts.max_scenes > 65536 ||
      opts.max_boxes < 1 || opts.memory_cap <= 0 || opts.arena_bytes < (1 << 20) || !(opts.delta >= 0) ||
      !(opts.min_sep >= 0) || opts.max_iter < 0 || !(opts.pairs_per_box >= 0) ||
      (opts.autotune != 0 && opts.autotune != 1))
    return CCD_EINVAL;
  if (cudaSetDevice(device) != cudaSuccess) return CCD_EINVAL;
  ccd_server *S = new (std::nothrow) ccd_server();
  if (!S) return CCD_ENOMEM;
  S->opts = opts;
  S->device = device;
  S->slot_mem = opts.memory_cap / opts.n_slots;
  ccd_opts co;
  ccd_default_opts(&co);
  co.delta = opts.delta;
  co.min_sep = opts.min_sep;
  co.max_iter = opts.max_iter;
  ccd_get_memory_model(&co, &S->mm);
  if (cudaHostAlloc(&S->arena, opts.arena_bytes, cudaHostAllocDefault) != cudaSuccess) {
    delete S;
    return CCD_ENOMEM;
  }
  S->arena_bytes = opts.arena_bytes;
  S->slots.resize(opts.n_slots);
  for (Slot &sl : S->slots) {
    // pair capacity from the slot's memory share for its largest batch
    ccd_opts so = co;
    const int64_t cap = ccd_pair_capacity_for(&co, S->slot_mem, opts.max_boxes, opts.max_scenes);
    const int64_t want = opts.pairs_per_box > 0 ? (int64_t)(opts.pairs_per_box * opts.max_boxes) : 4 * opts.max_boxes;
    so.pair_capacity = std::max<int64_t>(1 << 20, std::min<int64_t>(cap, want));
    int rc = ccd_create(&sl.ctx, &so, device);
    if (rc == CCD_OK && cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess) rc = CCD_ECUDA;
    if (rc) {
      ccd_server_destroy(S);
      return rc;
    }
  }
  S->sched = std::thread(scheduler, S);
  *out = S;
  return CCD_OK;
}

int ccd_server_destroy(ccd_server *S) {
  if (!S) return CCD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    // scenes handed out but never submitted would block the queue: drop them
    while (!S->queue.empty() && !S->queue.back()->submitted) S->queue.pop_back();
  }
  S->cv_sched.notify_all();
  if (S->sched.joinable()) S->sched.join();
  cudaSetDevice(S->device);
  for (Slot &sl : S->slots) {
    if (sl.stream) cudaStreamSynchronize(sl.stream);
    cudaFree(sl.staging);
    cudaFree(sl.V0);
    cudaFree(sl.V1);
    cudaFree(sl.toi);
    cudaFree(sl.E);
    cudaFree(sl.F);
    cudaFree(sl.offs);
    cudaFree(sl.desc);
    cudaFreeHost(sl.h_desc);
    cudaFreeHost(sl.h_toi);
    cudaFreeHost(sl.h_status);
    if (sl.stream) cudaStreamDestroy(sl.stream);
    if (sl.ctx) ccd_destroy(sl.ctx);
  }
  for (auto &kv : S->reqs) delete kv.second;
  for (Batch *b : S->inflight) delete b;
  if (S->arena) cudaFreeHost(S->arena);
  delete S;
  return CCD_OK;
}

int ccd_server_request(ccd_server *S, int64_t nV, int64_t nE, int64_t nF, double **V0, double **V1, int32_t **E,
                       int32_t **F, uint64_t *ticket) {
  if (!S || !V0 || !V1 || !E || !F || !ticket || nV < 0 || nE < 0 || nF < 0) return CCD_EINVAL;
  if (nV + nE + nF >= (1ll << 31)) return CCD_EINVAL;
  Block probe = make_block(0, nV, nE, nF);
  if (probe.bytes > S->arena_bytes / 2) return CCD_ENOMEM;
  if (nV + nE + nF > S->opts.max_boxes || est_bytes(S, nV + nE + nF, 1) > S->slot_mem) return CCD_ENOMEM;
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    if (S->stop) return CCD_EINVAL;
    // blocks never wrap: skip to the ring's start when the block would
    int64_t pos = S->head;
    const int64_t in_ring = pos % S->arena_bytes;
    if (in_ring + probe.bytes > S->arena_bytes) pos += S->arena_bytes - in_ring;
    if (pos + probe.bytes - S->tail <= S->arena_bytes) {
      Request *r = new (std::nothrow) Request();
      if (!r) return CCD_ENOMEM;
      r->id = S->next_id++;
      r->blk = make_block(pos, nV, nE, nF);
      S->head = pos + r->blk.bytes;
      S->queue.push_back(r);
      S->reqs[r->id] = r;
      unsigned char *base = S->arena + (pos % S->arena_bytes);
      *V0 = (double *)base;
      *V1 = (double *)(base + r->blk.oV1);
      *E = (int32_t *)(base + r->blk.oE);
      *F = (int32_t *)(base + r->blk.oF);
      *ticket = r->id;
      return CCD_OK;
    }
    S->cv_space.wait_for(lk, std::chrono::microseconds(100));
    finish_batches(S);
  }
}

int ccd_server_submit(ccd_server *S, uint64_t ticket) {
  if (!S) return CCD_EINVAL;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->reqs.find(ticket);
    if (it == S->reqs.end() || it->second->submitted) return CCD_EINVAL;
    it->second->submitted = true;
    it->second->t_submit = now_s();
    S->st.n_submitted += 1;
  }
  S->cv_sched.notify_one();
  return CCD_OK;
}

int ccd_server_submit_scene(ccd_server *S, int64_t nV, int64_t nE, int64_t nF, const double *V0, const double *V1,
                            const int32_t *E, const int32_t *F, uint64_t *ticket) {
  if (!S || !ticket || (nV > 0 && (!V0 || !V1)) || (nE > 0 && !E) || (nF > 0 && !F)) return CCD_EINVAL;
  double *a = nullptr, *b = nullptr;
  int32_t *e = nullptr, *f = nullptr;
  uint64_t t = 0;
  int rc = ccd_server_request(S, nV, nE, nF, &a, &b, &e, &f, &t);
  if (rc) return rc;
  if (nV > 0) {
    std::memcpy(a, V0, 3 * nV * sizeof(double));
    std::memcpy(b, V1, 3 * nV * sizeof(double));
  }
  if (nE > 0) std::memcpy(e, E, 2 * nE * sizeof(int32_t));
  if (nF > 0) std::memcpy(f, F, 3 * nF * sizeof(int32_t));
  rc = ccd_server_submit(S, t);
  if (rc) return rc;
  *ticket = t;
  return CCD_OK;
}


int ccd_server_wait(ccd_server *S, uint64_t ticket, double timeout_ms, double *toi, double *latency_ms) {
  if (!S || !toi) return CCD_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end() || !it->second->submitted) return CCD_EINVAL;
  Request *r = it->second;
  const double deadline = timeout_ms >= 0 ? now_s() + timeout_ms * 1e-3 : 0.0;
  while (!r->done) {
    finish_batches(S);
    if (r->done) break;
    if (timeout_ms >= 0 && now_s() >= deadline) return CCD_ETIMEOUT;
    S->cv_done.wait_for(lk, std::chrono::microseconds(50));
  }
  *toi = r->toi;
  if (latency_ms) *latency_ms = (r->t_done - r->t_submit) * 1e3;
  const int status = r->status;
  S->reqs.erase(it);
  delete r;
  return status;
}

int ccd_server_get_stats(ccd_server *S, ccd_server_stats *st) {
  if (!S || !st) return CCD_EINVAL;
  std::lock_guard<std::mutex> lk(S->mu);
  *st = S->st;
  return S->error;
}

}  // extern "C"
