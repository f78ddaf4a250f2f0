// pat_spectrum_noalloc: the zero-padded 2D real FFT of stage i for callers
// that cannot allocate device memory.
//
// The regular path (pat_stage_spectrum / the operators) keeps the row-pass
// intermediate T[slice][kx][y] in workspace that pat_plan_create allocates.
// This variant needs no plan: the intermediate lives in a file-scope static
// device array of fixed size, and the FFT twiddles in another, so a call
// performs no cudaMalloc / cudaFree and no allocating library routine.
//
// Who needs it: code that must not allocate on the device at the point of the
// call -- e.g. an application whose device memory is owned entirely by its own
// pool allocator, or a latency-critical loop where cudaMalloc (which can
// synchronise the device) is not allowed.
//
// Costs and rules (also in include/pat.h):
//   - every GPU that loads this module holds kScratchBytes (64 MiB) plus the
//     twiddle tables until the process exits;
//   - the first call on a device sets that device up (symbol addresses,
//     twiddle upload with a synchronous copy); make that first call before any
//     stream capture;
//   - all calls share the scratch array, which keeps the last call's
//     contents; nothing in it needs to start at zero (every element the
//     column pass reads is written by the row pass of the same call); calls
//     that overlap on the GPU (different streams, or threads) race on it.
#include <cmath>
#include <mutex>

#include "pat_internal.h"

namespace pat {
namespace {

constexpr size_t kScratchBytes = 64ull << 20;  // maximum row-pass intermediate
constexpr int kMaxDevices = 64;
// twiddles exp(-2 pi i k / P) for P = 16, 32, ..., 1024, concatenated
constexpr int kTwiddleTotal = 16 + 32 + 64 + 128 + 256 + 512 + 1024;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];
static __device__ __align__(256) float2 g_twiddles[kTwiddleTotal];

struct DeviceSetup {
  bool ready = false;
  void* scratch = nullptr;
  float2* twiddles = nullptr;
};
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

int twiddle_offset(int p) {
  int off = 0;
  for (int q = 16; q < p; q *= 2) off += q;
  return off;
}

// Once per device, with that device current: device addresses of the static
// arrays (their names are host-side stand-ins in host code) and the twiddles.
int setup_current_device(DeviceSetup** out) {
  int dev = 0;
  PAT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(PAT_ERR_UNSUPPORTED, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.ready) {
    void* scratch = nullptr;
    void* tw = nullptr;
    PAT_CUDA(cudaGetSymbolAddress(&scratch, g_scratch));
    PAT_CUDA(cudaGetSymbolAddress(&tw, g_twiddles));
    float2 host[kTwiddleTotal];
    const double pi = 3.14159265358979323846;
    for (int p = 16; p <= 1024; p *= 2) {
      const int off = twiddle_offset(p);
      for (int k = 0; k < p; ++k) {
        host[off + k].x = (float)std::cos(-2.0 * pi * k / p);
        host[off + k].y = (float)std::sin(-2.0 * pi * k / p);
      }
    }
    PAT_CUDA(cudaMemcpyToSymbol(g_twiddles, host, sizeof(host)));
    s.scratch = scratch;
    s.twiddles = static_cast<float2*>(tw);
    s.ready = true;
  }
  *out = &s;
  return PAT_OK;
}

bool pow2_in(int v) { return v >= 16 && v <= 1024 && (v & (v - 1)) == 0; }

}  // namespace
}  // namespace pat

using namespace pat;

extern "C" int pat_spectrum_noalloc(const float* in, int nx, int ny, int px, int py, int slices,
                                    void* out, pat_stream stream) {
  try {
    if (nx < 1 || ny < 1 || slices < 0) return fail(PAT_ERR_ARG, "nx, ny >= 1 and slices >= 0 required");
    if (!pow2_in(px) || !pow2_in(py))
      return fail(PAT_ERR_UNSUPPORTED, "px and py must be powers of two in [16, 1024]");
    if (px < 2 * nx - 1 || py < 2 * ny - 1)
      return fail(PAT_ERR_ARG, "padding too small for linear convolution: need px >= 2nx-1, py >= 2ny-1");
    const size_t need = (size_t)slices * (size_t)(px / 2 + 1) * (size_t)(ny + (ny & 1)) * 8;
    if (need > kScratchBytes)
      return fail(PAT_ERR_ARG, "pat_spectrum_noalloc: slices * (px/2 + 1) * ny_even * 8 = " +
                                   std::to_string(need) + " bytes exceeds its static scratch of " +
                                   std::to_string(kScratchBytes) + " bytes; use fewer slices per call");
    if (slices == 0) return PAT_OK;
    if (!in || !out) return fail(PAT_ERR_ARG, "in or out is NULL");
    // the scratch, the twiddles and the launch belong to the current device,
    // so both arrays must live there (there is no plan to tie them to)
    int dev = -1;
    PAT_CUDA(cudaGetDevice(&dev));
    const int din = device_of(in), dout = device_of(out);
    if (din < 0 || dout < 0) return fail(PAT_ERR_ARG, "pat_spectrum_noalloc takes device arrays");
    if (din != dev || dout != dev)
      return fail(PAT_ERR_ARG, "pat_spectrum_noalloc: in and out must be on the current device (" +
                                   std::to_string(dev) + "); they are on " + std::to_string(din) +
                                   " and " + std::to_string(dout));
    DeviceSetup* s = nullptr;
    int rc = setup_current_device(&s);
    if (rc != PAT_OK) return rc;
    // A transform-only view: grid, scratch and twiddles; nothing else is read.
    Plan view;
    view.L = Layout{};
    view.L.px = px;
    view.L.py = py;
    view.L.fp64 = false;
    view.T = s->scratch;
    view.twx = s->twiddles + twiddle_offset(px);
    view.twy = s->twiddles + twiddle_offset(py);
    PAT_CUDA(launch_spectrum(view, in, (int64_t)nx * ny, nx, ny, out,
                             (int64_t)(px / 2 + 1) * py, slices, (cudaStream_t)stream));
    return PAT_OK;
  } catch (...) {
    return fail(PAT_ERR_CUDA, "unexpected internal error");
  }
}
