// Allocation-free variant of the l1-ball projection entry point.
//
// Some callers cannot call cudaMalloc: code running inside a memory-pool or
// arena that owns all device allocations, a plug-in loaded into a host that
// forbids allocation after start-up, or a real-time loop that must not touch
// the allocator.  s3ttv_l1_ball_static serves them: it runs the same radix
// selection and soft-threshold kernels as s3ttv_l1_ball, but its scratch (the
// selection state and the histogram bins) is the file-scope array below, which
// every GPU that loads this library holds until the process exits.  The caller
// passes device buffers for the input and the output; nothing is allocated.
#include <cmath>
#include <mutex>

#include "s3ttv.h"
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

// Layout: [Scalars][pad to 256][kHistBins u32 counts][kHistBins double sums].
constexpr size_t kScalarsBytes = (sizeof(Scalars) + 255) & ~size_t(255);
constexpr size_t kCountBytes = sizeof(unsigned) * kHistBins;
constexpr size_t kSumBytes = sizeof(double) * kHistBins;
constexpr size_t kScratchBytes = kScalarsBytes + kCountBytes + kSumBytes;  // about 24.3 KB

static __device__ __align__(256) unsigned char g_l1_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_l1_scratch on the current device, looked up once per
// device.  In host code the symbol itself is only a host-side stand-in.
int scratch_address(int dev, unsigned char **out) {
  if (dev < 0 || dev >= kMaxDevices) return S3TTV_EUNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_l1_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return S3TTV_ECUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = static_cast<unsigned char *>(g_scratch_addr[dev]);
  return S3TTV_OK;
}

// Device memory of device dev itself, or managed memory.  Memory of another
// GPU is refused: the kernels run on dev, and without peer access such a
// pointer is not reachable from it.
bool on_device(const void *p, int dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeManaged || (at.type == cudaMemoryTypeDevice && at.device == dev);
}

}  // namespace
}  // namespace s3ttv

using namespace s3ttv;

extern "C" int s3ttv_l1_ball_static(const float *x, float *out, long long n, double radius, double *tau_out,
                                    void *stream) {
  if (n < 0 || !(radius >= 0) || !std::isfinite(radius)) return S3TTV_EINVAL;
  if (n > S3TTV_L1_STATIC_MAX_N) return S3TTV_ETOOBIG;
  if (n == 0) {
    if (tau_out) *tau_out = 0.0;
    return S3TTV_OK;
  }
  if (!x || !out) return S3TTV_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return S3TTV_ECUDA;
  }
  if (!on_device(x, dev) || !on_device(out, dev)) return S3TTV_EINVAL;
  unsigned char *base = nullptr;
  int rc = scratch_address(dev, &base);
  if (rc) return rc;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  Scalars *sc = reinterpret_cast<Scalars *>(base);
  unsigned *hcnt = reinterpret_cast<unsigned *>(base + kScalarsBytes);
  double *hsum = reinterpret_cast<double *>(base + kScalarsBytes + kCountBytes);
  // The array keeps whatever the previous call left: clear the bins and reset
  // the selection state before use.
  if (cudaMemsetAsync(hcnt, 0, kCountBytes + kSumBytes, st) != cudaSuccess) return S3TTV_ECUDA;
  if (launch_init_scalars(sc, radius, 0.0, st) != cudaSuccess) return S3TTV_ECUDA;
  L1Args la;
  la.x[0] = x;
  la.x[1] = x;
  la.n = n;
  la.nprob = 1;
  la.sc = sc;
  la.hcnt = hcnt;
  la.hsum = hsum;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  long long grid = (n + 255) / 256;
  const long long cap = (sms > 0 ? sms : 1) * 8ll;
  if (grid > cap) grid = cap;
  for (int level = 1; level <= 3; ++level) {
    if (launch_l1_hist(la, level, (int)grid, st) != cudaSuccess) return S3TTV_ECUDA;
    if (launch_l1_scan(la, level, st) != cudaSuccess) return S3TTV_ECUDA;
  }
  if (launch_soft_threshold(x, out, n, sc, 0, st) != cudaSuccess) return S3TTV_ECUDA;
  L1State state;
  if (cudaMemcpyAsync(&state, &sc->l1[0], sizeof(state), cudaMemcpyDeviceToHost, st) != cudaSuccess)
    return S3TTV_ECUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return S3TTV_ECUDA;
  if (tau_out) *tau_out = (double)state.tau;
  return S3TTV_OK;
}
