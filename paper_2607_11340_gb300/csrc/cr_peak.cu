// Peak-calibration kernels, timed by the caller in the same run as the solver: FP32 FMA chains
// (scalar and paired),
// special-function (MUFU sin/cos approximation) chains, FP64 FMA chains and a streaming copy.
// Each thread runs several independent dependency chains so that the pipes, not latency, bound it.
#include "cr_host.h"

namespace {

__global__ void __launch_bounds__(256) k_peak_ffma(float* out, int iters) {
  float a0 = threadIdx.x * 1e-3f, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3, a4 = a0 + 4, a5 = a0 + 5,
        a6 = a0 + 6, a7 = a0 + 7;
  const float m = 0.999999f, c = 1e-7f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = fmaf(a0, m, c); a1 = fmaf(a1, m, c); a2 = fmaf(a2, m, c); a3 = fmaf(a3, m, c);
      a4 = fmaf(a4, m, c); a5 = fmaf(a5, m, c); a6 = fmaf(a6, m, c); a7 = fmaf(a7, m, c);
    }
  }
  float s = a0 + a1 + a2 + a3 + a4 + a5 + a6 + a7;
  if (s == 12345.678f) out[threadIdx.x] = s;
}

// The same chains with the paired FP32 instruction (two independent FMAs per lane per instruction).
__global__ void __launch_bounds__(256) k_peak_ffma2(float* out, int iters) {
  const float b0 = threadIdx.x * 1e-3f;
  float2 a0 = make_float2(b0, b0 + 1), a1 = make_float2(b0 + 2, b0 + 3), a2 = make_float2(b0 + 4, b0 + 5),
         a3 = make_float2(b0 + 6, b0 + 7);
  const float2 m = make_float2(0.999999f, 0.999999f), c = make_float2(1e-7f, 1e-7f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      a0 = __ffma2_rn(a0, m, c); a1 = __ffma2_rn(a1, m, c); a2 = __ffma2_rn(a2, m, c); a3 = __ffma2_rn(a3, m, c);
    }
  }
  float s = a0.x + a0.y + a1.x + a1.y + a2.x + a2.y + a3.x + a3.y;
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_mufu(float* out, int iters) {
  float a0 = threadIdx.x * 1e-3f, a1 = a0 + 0.1f, a2 = a0 + 0.2f, a3 = a0 + 0.3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a0 = __sinf(a0); a1 = __cosf(a1); a2 = __sinf(a2); a3 = __cosf(a3);
    }
  }
  float s = a0 + a1 + a2 + a3;
  if (s == 12345.678f) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_dfma(double* out, int iters) {
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  const double m = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    }
  }
  double s = a0 + a1 + a2 + a3;
  if (s == 12345.678) out[threadIdx.x] = s;
}

// DFMA chains on one lane of every warp: how the FP64 pipe charges an instruction whose warp has
// a single active lane (the other lanes skip the loop).
__global__ void __launch_bounds__(256) k_peak_dfma_lane(double* out, int iters) {
  if ((threadIdx.x & 31) != 0) return;
  double a0 = threadIdx.x * 1e-3, a1 = a0 + 1, a2 = a0 + 2, a3 = a0 + 3;
  const double m = 0.9999999, c = 1e-9;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      a0 = fma(a0, m, c); a1 = fma(a1, m, c); a2 = fma(a2, m, c); a3 = fma(a3, m, c);
    }
  }
  double s = a0 + a1 + a2 + a3;
  if (s == 12345.678) out[threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) k_peak_copy(const float4* __restrict__ src, float4* __restrict__ dst, size_t n) {
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = src[i];
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

}  // namespace

extern "C" cr_status cr_peak_launch(int32_t kind, void* buf, size_t bytes, int32_t iters, double* ops_out,
                                    cr_stream stream) {
  using namespace crh;
  if (!buf || !ops_out || iters < 1 || bytes < 4096) return fail(CR_EINVAL, "cr_peak_launch: bad arguments");
  if (!aligned(buf, 16)) return fail(CR_EINVAL, "cr_peak_launch: buffer not 16-byte aligned");
  cudaStream_t s = stream_of(stream);
  const int blocks = sm_count() * 8, threads = 256;
  const double nthr = double(blocks) * threads;
  switch (kind) {
    case 0:
      k_peak_ffma<<<blocks, threads, 0, s>>>((float*)buf, iters);
      *ops_out = nthr * iters * 16 * 8 * 2.0;
      break;
    case 5:
      k_peak_ffma2<<<blocks, threads, 0, s>>>((float*)buf, iters);
      *ops_out = nthr * iters * 16 * 8 * 2.0;
      break;
    case 1:
      k_peak_mufu<<<blocks, threads, 0, s>>>((float*)buf, iters);
      *ops_out = nthr * iters * 8 * 4.0;
      break;
    case 2:
      k_peak_dfma<<<blocks, threads, 0, s>>>((double*)buf, iters);
      *ops_out = nthr * iters * 8 * 4 * 2.0;
      break;
    case 4:
      k_peak_dfma_lane<<<blocks, threads, 0, s>>>((double*)buf, iters);
      *ops_out = nthr / 32 * iters * 8 * 4 * 2.0;
      break;
    case 3: {
      size_t n = bytes / 2 / sizeof(float4);
      const float4* src = (const float4*)buf;
      float4* dst = (float4*)((char*)buf + n * sizeof(float4));
      k_peak_copy<<<sm_count() * 16, 256, 0, s>>>(src, dst, n);
      *ops_out = double(n) * sizeof(float4) * 2.0;
      break;
    }
    default:
      return fail(CR_EINVAL, "cr_peak_launch: kind %d", kind);
  }
  return check_launch("cr_peak_launch");
}
