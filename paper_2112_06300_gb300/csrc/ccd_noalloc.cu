// ccd_narrow_noalloc: the narrow phase without any device allocation.
//
// Some callers cannot call cudaMalloc at the point where they need a
// collision query: code that runs under a caching or pooled allocator they do
// not own, plug-ins whose host forbids allocation, or real-time loops that
// must not risk an allocation failure or the device-wide synchronisation a
// cudaMalloc/cudaFree may cause.  For them this entry point runs the same
// narrow-phase kernel as ccd_narrow with its scratch (control block, per-query
// flags and counters, interval ring) in one file-scope device array of fixed
// size.  Every GPU that loads this library holds that array until the process
// exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears what must start at zero (counters, status, the
// shared t*).  Calls that overlap on the GPU (two streams, or two host
// threads) race on it.

#include <cstring>
#include <mutex>

#include "ccd_common.cuh"
#include "ccd_kernels.cuh"

using namespace ccd;

namespace {

constexpr long long kMaxQueries = 1 << 16;       // vertex-face + edge-edge pairs per call
constexpr unsigned long long kRingCells = 1 << 14;
constexpr size_t kCtlBytes = (sizeof(DevCtl) + 255) / 256 * 256;
constexpr size_t kFlagsBytes = kMaxQueries * sizeof(uint32_t);
constexpr size_t kItersBytes = kMaxQueries * sizeof(unsigned long long);
constexpr size_t kRingBytes = kRingCells * sizeof(RingCell);
constexpr size_t kScratchBytes = kCtlBytes + kFlagsBytes + kItersBytes + kRingBytes;   // ~1.4 MB

static_assert(sizeof(DevCtl) % 8 == 0, "the control block is cleared as 8-byte words");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
  bool ready = false;
  unsigned char *base = nullptr;   // device address of g_scratch on this device
  int blocks = 0;
};

constexpr int kMaxDevices = 64;
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

__global__ void k_noalloc_init(unsigned char *base) {
  DevCtl *ctl = (DevCtl *)base;
  RingCell *ring = (RingCell *)(base + kCtlBytes + kFlagsBytes + kItersBytes);
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  if (tid < sizeof(DevCtl) / sizeof(unsigned long long))
    ((unsigned long long *)ctl)[tid] = 0;   // DevCtl is a whole number of 8-byte words
  for (unsigned long long i = tid; i < kRingCells; i += (unsigned long long)gridDim.x * blockDim.x)
    ring[i].seq = i;   // ring positions start at 0
}

__global__ void k_noalloc_reset(DevCtl *ctl) {
  ctl->status = CCD_OK;
  ctl->q_next = 0;
  ctl->pending = 0;
  ctl->toi_bits = 0x7FF0000000000000ull;
  ctl->n_intervals = ctl->n_exported = ctl->n_capped = ctl->queue_peak = 0;
  ctl->t_start = ctl->t_exhausted = ctl->t_end = 0;
  ctl->n_donated = 0;
  ctl->n_intervals_tail = 0;
  ctl->n_intervals_fp64 = 0;
  ctl->n_left = 0;
}

__global__ void k_noalloc_status(const DevCtl *ctl, int32_t *status) { *status = ctl->status; }

// One-time set-up on the current device: device address of the array,
// ring initialisation, persistent grid size.
int setup_device(int dev, cudaStream_t s, DeviceState **out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState &st = g_state[dev];
  if (!st.ready) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) return CCD_ECUDA;
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CCD_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow_setup, kNarrowThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    k_noalloc_init<<<64, 256, 0, s>>>((unsigned char *)p);
    if (cudaGetLastError() != cudaSuccess) return CCD_ECUDA;
    st.base = (unsigned char *)p;
    st.blocks = per_sm * sms;
    st.ready = true;
  }
  *out = &st;
  return CCD_OK;
}

}  // namespace

extern "C" int ccd_narrow_noalloc(const int32_t *vf, int64_t n_vf, const int32_t *ee, int64_t n_ee,
                                  const double *V0, const double *V1, int64_t nV, const int32_t *E, int64_t nE,
                                  const int32_t *F, int64_t nF, double delta, double min_sep, int64_t max_iter,
                                  int32_t mode, double *toi_vf, double *toi_ee, uint8_t *flags_vf,
                                  uint8_t *flags_ee, double *toi_min, int32_t *status, void *stream) {
  if (n_vf < 0 || n_ee < 0 || !toi_min || !status || (mode != 0 && mode != 1)) return CCD_EINVAL;
  if (n_vf + n_ee > kMaxQueries) return CCD_EINVAL;   // beyond the fixed scratch
  if (!(delta >= 0) || !(min_sep >= 0) || max_iter < 0) return CCD_EINVAL;
  if ((n_vf > 0 && (!vf || !F)) || (n_ee > 0 && (!ee || !E))) return CCD_EINVAL;
  if (nV < 0 || nE < 0 || nF < 0 || (nV > 0 && (!V0 || !V1))) return CCD_EINVAL;
  if (mode == 0 && ((n_vf > 0 && !toi_vf) || (n_ee > 0 && !toi_ee))) return CCD_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CCD_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  DeviceState *st = nullptr;
  int rc = setup_device(dev, s, &st);
  if (rc) return rc;
  unsigned char *base = st->base;
  DevCtl *ctl = (DevCtl *)base;
  k_noalloc_reset<<<1, 1, 0, s>>>(ctl);
  NarrowArgs A;
  std::memset(&A, 0, sizeof(A));
  A.ctl = ctl;
  A.vf = vf;
  A.ee = ee;
  A.n_vf = n_vf;
  A.n_ee = n_ee;
  A.counts_from_ctl = 0;
  A.V0 = V0;
  A.V1 = V1;
  A.nV = nV;
  A.E = E;
  A.F = F;
  A.delta = delta;
  A.min_sep = min_sep;
  A.max_iter = max_iter;
  A.mode = mode;
  A.budget = 64;
  A.no_zero = 0;
  A.only_if_rerun = 0;
  A.qrec = nullptr;   // no record buffer: lanes set their queries up themselves
  A.rec_stride = 0;
  A.n_scenes = 0;
  A.voff = nullptr;
  A.toi_scene = nullptr;
  A.qsid = nullptr;
  A.toi_vf_bits = mode == 0 ? (unsigned long long *)toi_vf : nullptr;
  A.toi_ee_bits = mode == 0 ? (unsigned long long *)toi_ee : nullptr;
  A.qflags = (uint32_t *)(base + kCtlBytes);
  A.qiters = (unsigned long long *)(base + kCtlBytes + kFlagsBytes);
  A.ring = (RingCell *)(base + kCtlBytes + kFlagsBytes + kItersBytes);
  A.ring_mask = kRingCells - 1;
  k_narrow_setup<<<st->blocks, kNarrowThreads, 0, s>>>(A);
  if (mode == 0 && n_vf + n_ee > 0)
    k_flags_out<<<64, 256, 0, s>>>(A.qflags, n_vf, n_ee, flags_vf, flags_ee, ctl);
  if (cudaMemcpyAsync(toi_min, &ctl->toi_bits, sizeof(double), cudaMemcpyDeviceToDevice, s) != cudaSuccess)
    return CCD_ECUDA;
  k_noalloc_status<<<1, 1, 0, s>>>(ctl, status);
  return cudaGetLastError() == cudaSuccess ? CCD_OK : CCD_ECUDA;
}
