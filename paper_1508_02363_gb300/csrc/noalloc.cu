// Allocation-free 2-D DFT: dbar_fft2_noalloc.
//
// Some callers cannot allocate device memory at the point where they need a
// transform: kernels-only plugins whose host runtime owns every byte of device
// memory through its own pool (a cudaMalloc there would bypass the pool's
// accounting or fail against its reservation), and latency-critical loops
// that forbid allocator calls (cudaMalloc/cudaFree can synchronise the device
// and take milliseconds).  For them
// this entry point runs the same row and column transform kernels as
// dbar_fft2, but keeps its intermediate field and its twiddle tables in
// global arrays that belong to the library image itself, so a call allocates
// nothing.
//
// Costs and rules of that choice:
//  * Every GPU that loads the library holds kScratchBytes (32 MiB: one 2048^2
//    complex64 field, the largest grid's FP32 transform) plus the twiddle
//    tables (about 100 KiB) until the process exits.
//  * All calls share the one scratch array: calls that overlap on the GPU
//    (different host threads, or different streams without ordering) race.
//  * The first call on a device copies the twiddle tables there and looks up
//    the arrays' device addresses (cudaMemcpyToSymbol, cudaGetSymbolAddress)
//    with that device current.
//  * Each call returns after the caller's stream has drained (it ends with a
//    cudaStreamSynchronize, like the library's other entry points).
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/dbar.h"
#include "launch.cuh"

using namespace dbar;

namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;  // 32 MiB
constexpr int kMinLog = 5, kMaxLog = 11;              // N = 32 .. 2048
constexpr int kTableLen = (1 << (kMaxLog + 1)) - (1 << kMinLog);  // sum of all supported N
constexpr int kMaxDevices = 64;

// the intermediate (row-transformed) field; fully overwritten by the row pass
// before the column pass reads it, so nothing in it must start at zero
__device__ __align__(256) unsigned char g_scratch[kScratchBytes];
// e^{-2 pi i t/N} for every supported N, table of size N at offset N - 32
__device__ __align__(256) cx<double> g_tw64[kTableLen];
__device__ __align__(256) cx<float> g_tw32[kTableLen];

struct DeviceState {
  bool ready = false;
  void* scratch = nullptr;
  cx<double>* tw64 = nullptr;
  cx<float>* tw32 = nullptr;
};
std::mutex g_mutex;
DeviceState g_state[kMaxDevices];
// host staging for the one-time table upload (static storage: no heap use)
cx<double> h_tw64[kTableLen];
cx<float> h_tw32[kTableLen];

dbar_status setup(int dev, DeviceState** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (dev < 0 || dev >= kMaxDevices) return dbar_internal_fail(DBAR_ECUDA, "device ordinal out of range");
  DeviceState& d = g_state[dev];
  if (!d.ready) {
    for (int l = kMinLog; l <= kMaxLog; ++l) {
      const int N = 1 << l, off = N - (1 << kMinLog);
      for (int t = 0; t < N; ++t) {
        const double ang = 2.0 * M_PI * (double)t / (double)N;
        h_tw64[off + t] = mkc(std::cos(ang), -std::sin(ang));
        h_tw32[off + t] = mkc((float)std::cos(ang), (float)-std::sin(ang));
      }
    }
    cudaError_t e = cudaMemcpyToSymbol(g_tw64, h_tw64, sizeof(h_tw64));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_tw32, h_tw32, sizeof(h_tw32));
    if (e == cudaSuccess) e = cudaGetSymbolAddress(&d.scratch, g_scratch);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tw64, g_tw64);
    if (e == cudaSuccess) e = cudaGetSymbolAddress((void**)&d.tw32, g_tw32);
    if (e != cudaSuccess)
      return dbar_internal_fail(DBAR_ECUDA, std::string("allocation-free FFT set-up: ") + cudaGetErrorString(e));
    d.ready = true;
  }
  *out = &d;
  return DBAR_OK;
}

template <typename T>
dbar_status run(int N, int nk, const void* in, void* out, int sign, void* scratch, const cx<T>* tw,
                cudaStream_t st) {
  PassArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.g = make_geo<T>(N);
  a.sx1 = a.sy1 = N;  // every column and row
  a.tw = tw + (N - (1 << kMinLog));
  a.in = reinterpret_cast<const cx<T>*>(in);
  a.in_ss = (long long)N * N;
  a.out = scratch;
  a.out_ss = (long long)N * N;
  cudaError_t e = sign < 0 ? launch_pass_c<T, T, PC_FWD>(a, nk, st) : launch_pass_c<T, T, PC_INV>(a, nk, st);
  if (e == cudaSuccess) {
    a.in = reinterpret_cast<const cx<T>*>(scratch);
    a.out = out;
    e = sign < 0 ? launch_pass_b<T, PB_FWD>(a, nk, st) : launch_pass_b<T, PB_INV>(a, nk, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return dbar_internal_fail(DBAR_ECUDA, std::string("dbar_fft2_noalloc: ") + cudaGetErrorString(e));
  return DBAR_OK;
}

}  // namespace

extern "C" dbar_status dbar_fft2_noalloc(int N, int nk, const void* in, void* out, int sign, int fp32,
                                         void* stream) {
  if (N < (1 << kMinLog) || N > (1 << kMaxLog) || (N & (N - 1)))
    return dbar_internal_fail(DBAR_EINVAL, "dbar_fft2_noalloc: N must be a power of two in [32, 2048]");
  if (nk < 0) return dbar_internal_fail(DBAR_EINVAL, "dbar_fft2_noalloc: nk < 0");
  if (sign != 1 && sign != -1) return dbar_internal_fail(DBAR_EINVAL, "dbar_fft2_noalloc: sign must be +1 or -1");
  if (nk == 0) return DBAR_OK;
  if (!in || !out) return dbar_internal_fail(DBAR_EINVAL, "dbar_fft2_noalloc: NULL pointer");
  const size_t bytes = (size_t)nk * N * N * (fp32 ? sizeof(cx<float>) : sizeof(cx<double>));
  if (bytes > kScratchBytes)
    return dbar_internal_fail(DBAR_EINVAL, "dbar_fft2_noalloc: nk*N*N fields exceed the 32 MiB scratch "
                                           "(at most 2M complex128 or 4M complex64 values per call)");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return dbar_internal_fail(DBAR_ECUDA, "dbar_fft2_noalloc: no device");
  DeviceState* d = nullptr;
  dbar_status s = setup(dev, &d);
  if (s != DBAR_OK) return s;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  return fp32 ? run<float>(N, nk, in, out, sign, d->scratch, d->tw32, st)
              : run<double>(N, nk, in, out, sign, d->scratch, d->tw64, st);
}
