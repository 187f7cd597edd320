// gb_rhs_noalloc: the GB_MIXED right-hand side with its scratch in a static
// device array, for callers that must not have the library allocate device
// memory on their behalf (see include/gb.h).
//
// The regular gb_rhs of a GB_MIXED solver converts the caller's canonical q
// into the kernel's internal layout and the result back, through two of the
// solver's own field buffers.  This variant does the same through
// g_rhs_scratch, a file-scope array that every GPU loading the library holds
// until the process exits; it calls no cudaMalloc or cudaFree.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdio>
#include <mutex>

#include "gb.h"
#include "gb_internal.h"

namespace {

// 4 Mi floats = 16 MiB per device: room for the internal copies of q and F of
// up to 2 Mi floats each (N = 4: 22795 elements; N = 3: 34952; N = 2: 58254).
constexpr size_t kScratchFloats = size_t(4) << 20;
static __device__ __align__(256) float g_rhs_scratch[kScratchFloats];

// Device address of g_rhs_scratch per device ordinal, looked up on the first
// call for a solver of that device (with that device current).  In host code
// g_rhs_scratch itself only names a host-side stand-in; kernels must be given
// this address.  The table is read and filled under g_scratch_mu, so first
// calls from several host threads do not race.
constexpr int kMaxDevices = 64;
float *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

}  // namespace

extern "C" int gb_rhs_noalloc(gb_solver *s, double t, const void *q_dev, void *F_dev) {
  if (!s) return GB_EINVAL;
  if (!q_dev || !F_dev) return gb::set_solver_error(s, GB_EINVAL, "gb_rhs_noalloc: NULL q or F");
  if (!std::isfinite(t)) return gb::set_solver_error(s, GB_EINVAL, "gb_rhs_noalloc: t must be finite");
  gb::StageArgs a;
  const int32_t *perm = nullptr;
  int N = 0, Np = 0, precision = 0, num_sms = 1, sdev = 0;
  int64_t K = 0;
  void *stream = nullptr;
  if (gb::rhs_launch_view(s, t, &a, &perm, &N, &K, &Np, &precision, &stream, &num_sms, &sdev) != GB_OK)
    return gb::set_solver_error(s, GB_EINVAL, "gb_rhs_noalloc: not available for dim = 3 solvers");
  if (precision != GB_MIXED)
    return gb::set_solver_error(s, GB_EINVAL, "gb_rhs_noalloc: only GB_MIXED solvers use scratch; call gb_rhs");
  const int S = gb::mixed_stride(N);
  const size_t half = (size_t)((K + 15) / 16) * 16 * (size_t)S;   // internal layout, tiles of 16 elements
  if (2 * half > kScratchFloats) {
    char msg[200];
    snprintf(msg, sizeof(msg),
             "gb_rhs_noalloc: this mesh needs %zu floats of scratch but the static array holds %zu "
             "(at N = %d at most %lld elements); use gb_rhs",
             2 * half, kScratchFloats, N, (long long)(kScratchFloats / 2 / S / 16 * 16));
    return gb::set_solver_error(s, GB_EINVAL, msg);
  }
  // the scratch used is the copy of the array on the solver's device; cudaGetSymbolAddress
  // answers for the current device, so the solver's device must be the current one
  int dev = 0;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return gb::set_solver_error(s, GB_ECUDA, cudaGetErrorString(ce));
  if (dev != sdev) {
    char msg[160];
    snprintf(msg, sizeof(msg), "gb_rhs_noalloc: the solver lives on device %d but device %d is current; "
             "make the solver's device current first", sdev, dev);
    return gb::set_solver_error(s, GB_EINVAL, msg);
  }
  if (sdev < 0 || sdev >= kMaxDevices) return gb::set_solver_error(s, GB_EINVAL, "gb_rhs_noalloc: device ordinal >= 64");
  float *q_int = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu);
    if (!g_scratch_addr[sdev]) {
      float *p = nullptr;
      ce = cudaGetSymbolAddress((void **)&p, g_rhs_scratch);
      if (ce != cudaSuccess || !p)
        return gb::set_solver_error(s, GB_ECUDA, "gb_rhs_noalloc: cudaGetSymbolAddress of the scratch array failed");
      g_scratch_addr[sdev] = p;
    }
    q_int = g_scratch_addr[sdev];
  }
  float *F_int = q_int + half;
  cudaStream_t st = (cudaStream_t)stream;
  // the previous call's contents stay in the array: clear the padding slots and the
  // tail rows of the last tile that the conversion below does not write
  ce = cudaMemsetAsync(q_int, 0, half * sizeof(float), st);
  if (ce != cudaSuccess) return gb::set_solver_error(s, GB_ECUDA, cudaGetErrorString(ce));
  int rc = gb::launch_relayout(q_dev, nullptr, false, true, q_int, perm, K, Np, S, 0.0, st);
  if (rc == 0) {
    a.qin = q_int;
    a.qn = q_int;
    a.Fout = F_int;
    rc = gb::launch_stage_mixed(N, a, st, num_sms);
  }
  if (rc == 0) rc = gb::launch_relayout(nullptr, F_dev, false, false, F_int, perm, K, Np, S, 0.0, st);
  if (rc != 0) return gb::set_solver_error(s, GB_ECUDA, cudaGetErrorString((cudaError_t)rc));
  return GB_OK;
}
