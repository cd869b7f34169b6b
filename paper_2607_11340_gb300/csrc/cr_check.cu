// Elementwise runs of device helpers whose numerics the solvers rely on, so that they can be checked
// against reference results: CR_CHECK_RECIP gives recip_nr(in[i]) (FP64 reciprocal by Newton-Raphson
// from the single-precision approximation); CR_CHECK_SIN / CR_CHECK_COS the FP64 sine / cosine of
// the kinematics.
#include "cr_device.cuh"
#include "cr_host.h"

namespace {
__global__ void k_check_recip(const double* in, double* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = crk::recip_nr(in[i]);
}
__global__ void k_check_sincos(const double* in, double* out, int64_t n, int cosine) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s, c;
  crk::c_sincos(in[i], &s, &c);
  out[i] = cosine ? c : s;
}
}  // namespace

extern "C" cr_status cr_device_check(int32_t which, const double* in, double* out, int64_t n, cr_stream stream) {
  using namespace crh;
  if (n < 0) return fail(CR_EINVAL, "cr_device_check: n < 0");
  if (n == 0) return CR_OK;
  cr_status st;
  if ((st = check_ptr(in, 8, "in", true)) || (st = check_ptr(out, 8, "out", true))) return st;
  cudaStream_t s = stream_of(stream);
  switch (which) {
    case CR_CHECK_RECIP:
      k_check_recip<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n);
      return check_launch("cr_device_check");
    case CR_CHECK_SIN:
    case CR_CHECK_COS:
      k_check_sincos<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(in, out, n, which == CR_CHECK_COS);
      return check_launch("cr_device_check");
    default:
      return fail(CR_EINVAL, "cr_device_check: unknown helper %d", which);
  }
}
