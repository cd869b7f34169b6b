// cr_solve_ik_static: beam-search IK for callers that cannot allocate device memory.
//
// Some callers may not call cudaMalloc at all. One example is a robot's real-time control loop that
// reserves its resources at start-up, because an allocation there can block or synchronise the
// device at a moment the loop cannot afford. Another is a host program that hands all device memory
// out of its own fixed pool. This entry point needs no workspace from the caller: its scratch is
// one file-scope device array, CR_STATIC_WS_BYTES bytes, that every GPU loading the library keeps
// until the process exits. The caller still owns the targets and the outputs.
//
// The host cannot use the array's name as a device address, so the address comes from
// cudaGetSymbolAddress, resolved once per device with that device current. That happens on the first
// call on each device, so the first call should come before any stream capture. Every call shares
// the one array and overwrites it; the status word at its start is cleared on every call. Calls that
// overlap on the GPU (different streams, or different host threads, on the same device) race on the
// array and must be serialised by the caller.
#include <mutex>

#include "cr_host.h"

namespace {

__device__ __align__(256) unsigned char g_cr_static_ws[CR_STATIC_WS_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

cr_status static_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return crh::fail(CR_ECUDA, "cr_solve_ik_static: cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return crh::fail(CR_EINVAL, "cr_solve_ik_static: device %d unsupported", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_cr_static_ws);
    if (e != cudaSuccess || !p)
      return crh::fail(CR_ECUDA, "cr_solve_ik_static: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CR_OK;
}

}  // namespace

extern "C" size_t cr_static_workspace_capacity(void) { return CR_STATIC_WS_BYTES; }

extern "C" cr_status cr_solve_ik_static(const cr_robot* robot, const cr_scene* scene, const cr_task* task,
                                        const cr_ik_params* prm, double* u_out, double* cost_out,
                                        double* pos_err, double* rot_err, uint8_t* success, cr_stream stream) {
  cr_status st;
  if ((st = crh::check_robot(robot))) return st;
  if (!task || !prm) return crh::fail(CR_EINVAL, "cr_solve_ik_static: NULL task or params");
  if (task->n_targets < 0) return crh::fail(CR_EINVAL, "cr_solve_ik_static: n_targets < 0");
  size_t need = cr_ik_workspace_size(robot, task->n_targets, prm);
  if (need > CR_STATIC_WS_BYTES)
    return crh::fail(CR_EINVAL, "cr_solve_ik_static: %lld targets need %zu bytes of scratch, the static array holds %zu",
                     (long long)task->n_targets, need, (size_t)CR_STATIC_WS_BYTES);
  void* ws = nullptr;
  if ((st = static_address(&ws))) return st;
  return cr_solve_ik(robot, scene, task, prm, u_out, cost_out, pos_err, rot_err, success, ws, CR_STATIC_WS_BYTES,
                     stream);
}
