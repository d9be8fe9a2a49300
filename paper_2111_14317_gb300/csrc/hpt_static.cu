// hpt_step_static: the Euler-Newton step of hpt_step with its scratch memory
// taken from a fixed array compiled into the library instead of from
// cudaMalloc.  It exists for callers that must not allocate device memory
// while they run: applications that hand all device memory to their own
// allocator or pool up front and forbid libraries from allocating behind it,
// code with a fixed device-memory budget that must not grow at run time, and
// loops where the implicit device synchronisation of cudaMalloc/cudaFree is
// unacceptable.  The paper has no counterpart of this entry point.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code only holds a stand-in for its name, so the device address
// is fetched once per device with cudaGetSymbolAddress (with that device
// current) and cached.  All calls on a device share the array and it keeps
// the last call's contents; the only value that must start at zero (the FP64
// re-solve counter) is cleared by every solve launch.
#include <algorithm>
#include <mutex>

#include "hpt_internal.h"

namespace hpt {
namespace {

constexpr size_t kStaticScratchBytes = (size_t)32 << 20;   // 32 MiB
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mutex;
void* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the array on `dev` (the current device); fetched on the
// first call on that device.
hpt_status static_scratch(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return HPT_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
    if (e != cudaSuccess || !ptr) {
      set_error("cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      return HPT_ECUDA;
    }
    g_static_ptr[dev] = ptr;
  }
  *out = g_static_ptr[dev];
  return HPT_OK;
}

}  // namespace
}  // namespace hpt

using namespace hpt;

extern "C" hpt_status hpt_step_static(hpt_system s, int64_t p, const hpt_paths* S, int32_t nsteps,
                                      const hpt_params* prm, void* stream) {
  if (!s) { set_error("NULL handle"); return HPT_EINVAL; }
  if (!prm || !S || p < 0 || nsteps < 0) { set_error("bad params, state, p or nsteps"); return HPT_EINVAL; }
  if (s->proj) { set_error("hpt_step_static: the projective form is not supported"); return HPT_ENOTSUP; }
  const int n = s->n;
  const size_t cs = s->prec == HPT_FP64 ? 16 : 8;
  // layout: [re-solve counter, 256 B][re-solve list, p int64][extended
  // Jacobian of ceil(p/128)*128 paths]; max_p bounds 511 + 8p + (p+127) B
  const size_t per_path = (size_t)n * (n + 2) * cs + sizeof(int64_t);
  const size_t jac = (size_t)n * (n + 2) * cs;
  const int64_t max_p = (int64_t)((kStaticScratchBytes - 511 - 127 * jac) / per_path);
  if (p > max_p) {
    set_error("hpt_step_static: p=%lld exceeds the static scratch limit of %lld paths for n=%d "
              "(%zu bytes per path in %zu bytes)", (long long)p, (long long)max_p, n, per_path,
              kStaticScratchBytes);
    return HPT_ERANGE;
  }
  if (p == 0 || nsteps == 0) return HPT_OK;
  hpt_status rc0 = check_params(prm);
  if (rc0 == HPT_OK) rc0 = check_state(S, prm);
  if (rc0) return rc0;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != s->device) {
    set_error("the handle belongs to device %d, current device is %d", s->device, dev);
    return HPT_EINVAL;
  }
  void* base = nullptr;
  hpt_status rc = static_scratch(dev, &base);
  if (rc) return rc;
  // rounds of at most kChunk paths, as hpt_step runs them, so that no launch
  // is larger than the ones hpt_step makes; the scratch holds one round
  const int64_t chunk = std::min<int64_t>(p, kChunk);
  int32_t* redo_count = (int32_t*)base;
  int64_t* redo_list = (int64_t*)((char*)base + 256);
  void* ext = (char*)base + 256 + ((size_t)chunk * sizeof(int64_t) + 255) / 256 * 256;
  cudaStream_t st = (cudaStream_t)stream;
  for (int r = 0; r < nsteps; ++r) {
    for (int64_t q0 = 0; q0 < p; q0 += chunk) {
      const int64_t cnt = std::min(chunk, p - q0);
      const hpt_paths sub = offset_paths(*S, q0, n, cs);
      EvalOut out;
      out.ext = ext;
      cudaError_t e = s->prec == HPT_FP64 ? launch_eval_fp64(s, cnt, sub.y, sub.tau, 0, out, st)
                                          : launch_eval_mixed(s, cnt, sub.y, sub.tau, 0, out, st);
      if (e != cudaSuccess) {
        set_error("evaluation launch: %s", cudaGetErrorString(e));
        return HPT_ECUDA;
      }
      StepArgs a;
      a.n = n;
      a.p = cnt;
      a.ext = ext;
      a.st = sub;
      a.prm = *prm;
      a.err = s->d_err;
      a.redo_count = redo_count;
      a.redo_list = redo_list;
      e = launch_solve_update(s, a, st);
      if (e != cudaSuccess) {
        set_error("solve launch: %s", cudaGetErrorString(e));
        return HPT_ECUDA;
      }
    }
  }
  return HPT_OK;
}
