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
// contents.  Each call first puts all of it that the kernel reads back into
// the state of a first call: counters, status and the shared t* cleared, the
// ring's positions zeroed and every ring cell's sequence number rewritten.  So
// nothing an earlier call left behind -- finished, failed with CCD_ETIMEOUT,
// or cut off with intervals still in the ring -- reaches the next call.
// Calls that overlap on the GPU (two streams, or two host threads) race on it.
//
// Deliberate differences from ccd_narrow: the interval ring holds 2^14 cells
// (ccd_narrow: 2^21 by default), so fewer subtrees can wait in it during the
// tail (a hand-off that does not fit stays with its lane; results are the
// same); the hand-off budget is ccd_narrow's default (16).

#include <cstddef>
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
static_assert(offsetof(DevCtl, toi_bits) % 8 == 0, "t* is one 8-byte word of the control block");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceState {
  bool ready = false;
  int blocks = 0;                  // persistent grid of the narrow kernel
};

constexpr int kMaxDevices = 64;
DeviceState g_state[kMaxDevices];
std::mutex g_mutex;

// Every call: the control block back to zero (t* to +inf), the ring's
// positions to 0 and each cell's sequence number to its index, as for the
// first call on the device.
__global__ void k_noalloc_reset(unsigned char *base) {
  DevCtl *ctl = (DevCtl *)base;
  RingCell *ring = (RingCell *)(base + kCtlBytes + kFlagsBytes + kItersBytes);
  const unsigned long long tid = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x;
  // DevCtl is a whole number of 8-byte words; one thread writes each
  constexpr unsigned long long kToiWord = offsetof(DevCtl, toi_bits) / sizeof(unsigned long long);
  if (tid < sizeof(DevCtl) / sizeof(unsigned long long))
    ((unsigned long long *)ctl)[tid] = tid == kToiWord ? 0x7FF0000000000000ull : 0ull;
  for (unsigned long long i = tid; i < kRingCells; i += (unsigned long long)gridDim.x * blockDim.x)
    ring[i].seq = i;
}

__global__ void k_noalloc_status(const DevCtl *ctl, int32_t *status) { *status = ctl->status; }

// Set-up on the current device: the persistent grid size, once per device,
// and the array's device address.  In host code g_scratch names a host-side
// stand-in, not device memory, so the kernels get the address that
// cudaGetSymbolAddress returns for the current device.  The address is looked
// up again on every call (a host-side table lookup, no device work), so a
// cudaDeviceReset between calls, which reloads the module, is handled.
int setup_device(int dev, DeviceState **out, unsigned char **base) {
  void *p = nullptr;
  if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) return CCD_ECUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  DeviceState &st = g_state[dev];
  if (!st.ready) {
    int sms = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CCD_ECUDA;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_narrow_setup, kNarrowThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    st.blocks = per_sm * sms;
    st.ready = true;
  }
  *out = &st;
  *base = (unsigned char *)p;
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
  unsigned char *base = nullptr;
  int rc = setup_device(dev, &st, &base);
  if (rc) return rc;
  DevCtl *ctl = (DevCtl *)base;
  k_noalloc_reset<<<64, 256, 0, s>>>(base);
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
  A.budget = 16;   // ccd_narrow's default hand-off budget
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
