// lbm_conserved_noalloc: the global mass / momentum / energy sums of a dense
// f array, for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc (or cannot hand this library a
// workspace): code that runs while a stream is being captured into a CUDA
// graph, where allocation calls are not permitted; host frameworks whose
// allocator owns all of device memory and grants none to libraries; and
// monitoring or checkpoint hooks that must not change the device's memory
// footprint.  This entry point needs no workspace: its per-block partial
// sums live in one file-scope __device__ array (kNoallocBlocks x 8 doubles,
// 256 KiB) that every GPU which loads this library holds until the process
// exits.  The caller passes the input f and the output only.
//
// The array is shared by every call on a device and keeps the last call's
// contents; the completion counter is cleared at the start of each call.
// Calls whose kernels overlap on the same GPU (for example, calls issued on
// two streams without ordering between them) race on the array and give wrong
// sums.  The first call on each device looks up the array's device address
// (cudaGetSymbolAddress with that device current) and loads both kernel
// instantiations; make that first call before any stream capture begins.
// The address is kept together with the unique id of the CUDA context it came
// from: after cudaDeviceReset (or any teardown of the device's context) the
// next call finds a new context id and looks the address up again, so no
// call uses an address of a destroyed context.  With the output in host
// memory the call synchronises its stream, which a stream under capture
// cannot do: such calls are refused (LBM_EINVAL) before anything is queued.
#include <cmath>
#include <mutex>

#include "lbm_internal.cuh"

namespace lbm {
namespace {

constexpr int kNoallocThreads = 256;
constexpr int kNoallocCellsPerThread = 32;
constexpr long long kNoallocCellsPerBlock = (long long)kNoallocThreads * kNoallocCellsPerThread;  // 8192
constexpr int kNoallocBlocks = 4096;
constexpr long long kNoallocMaxCells = kNoallocBlocks * kNoallocCellsPerBlock;  // 33,554,432
constexpr int kMaxDevices = 64;

// Scratch: per-block partials (8 doubles each: 5 sums and padding), then the
// completion counter and the result slot used when the output is on the host.
struct NoallocScratch {
  double partials[kNoallocBlocks * 8];
  double result[8];
  unsigned counter;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

struct Consts {
  double c1, s, eta0sq, c1sq, c2sq;
};

// Block b sums cells [b * 8192, (b + 1) * 8192) of the dense f (x fastest),
// thread t taking cells b*8192 + t + 256*j; the last block to finish adds the
// partials in block order.  Same double-precision moments as lbm_conserved.
template <typename R>
__global__ void __launch_bounds__(kNoallocThreads)
    noalloc_conserved_kernel(const R* __restrict__ f, long long n, Consts m, NoallocScratch* __restrict__ scr,
                             double* __restrict__ out) {
  __shared__ double sh[5][kNoallocThreads];
  __shared__ bool last;
  double acc[5] = {0, 0, 0, 0, 0};
  const long long first = (long long)blockIdx.x * kNoallocCellsPerBlock;
  for (int j = 0; j < kNoallocCellsPerThread; ++j) {
    const long long k = first + threadIdx.x + (long long)j * kNoallocThreads;
    if (k >= n) break;
    double v[NV];
#pragma unroll
    for (int i = 0; i < NV; ++i) v[i] = (double)f[i * n + k];
    const double sa = ((v[1] + v[2]) + (v[3] + v[4])) + (v[5] + v[6]);
    const double sd = ((v[7] + v[8]) + (v[9] + v[10])) + ((v[11] + v[12]) + (v[13] + v[14]));
    acc[0] += v[0] + sa + sd;
    acc[1] += m.c1 * (v[1] - v[2]) + m.s * (((v[7] + v[8]) + (v[9] + v[10])) - ((v[11] + v[12]) + (v[13] + v[14])));
    acc[2] += m.c1 * (v[3] - v[4]) + m.s * (((v[7] + v[8]) + (v[11] + v[12])) - ((v[9] + v[10]) + (v[13] + v[14])));
    acc[3] += m.c1 * (v[5] - v[6]) + m.s * (((v[7] + v[9]) + (v[11] + v[13])) - ((v[8] + v[10]) + (v[12] + v[14])));
    acc[4] += m.eta0sq * v[0] + m.c1sq * sa + m.c2sq * sd;
  }
#pragma unroll
  for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] = acc[q];
  __syncthreads();
  for (int w = kNoallocThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
#pragma unroll
      for (int q = 0; q < 5; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
#pragma unroll
    for (int q = 0; q < 5; ++q) scr->partials[blockIdx.x * 8 + q] = sh[q][0];
    __threadfence();
    last = atomicAdd(&scr->counter, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double s[5] = {0, 0, 0, 0, 0};
    for (unsigned b = 0; b < gridDim.x; ++b) {
#pragma unroll
      for (int q = 0; q < 5; ++q) s[q] += ((volatile double*)scr->partials)[b * 8 + q];
    }
#pragma unroll
    for (int q = 0; q < 5; ++q) out[q] = s[q];
    scr->counter = 0u;
  }
}

std::mutex g_setup_mutex;
NoallocScratch* g_scratch_ptr[kMaxDevices] = {nullptr};
unsigned long long g_scratch_ctx[kMaxDevices] = {0};  // id of the context the address belongs to

// cuCtxGetCurrent / cuCtxGetId through the runtime's driver entry point (no -lcuda).
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

cudaError_t current_context_id(unsigned long long* id) {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  if (!get_current || !get_id) {
    void* p = nullptr;
    void* q = nullptr;
    cudaDriverEntryPointQueryResult r1, r2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &r1) != cudaSuccess ||
        r1 != cudaDriverEntryPointSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &q, 12000, cudaEnableDefault, &r2) != cudaSuccess ||
        r2 != cudaDriverEntryPointSuccess)
      return cudaErrorNotSupported;
    get_current = (CtxGetCurrentFn)p;
    get_id = (CtxGetIdFn)q;
  }
  CUcontext ctx = nullptr;
  if (get_current(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  return get_id(ctx, id) == CUDA_SUCCESS ? cudaSuccess : cudaErrorDeviceUninitialized;
}

// Device address of the scratch array on the current device.  Looked up
// (cudaGetSymbolAddress with that device current) on the first call and
// again whenever the device's context has changed since; the set-up also
// loads both kernel instantiations, so a later call enqueues launches only.
// The caller has made a runtime call on this device already, so its primary
// context is current.
cudaError_t scratch_for_current_device(NoallocScratch** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  unsigned long long ctx = 0;
  e = current_context_id(&ctx);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev] || g_scratch_ctx[dev] != ctx) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    cudaFuncAttributes fa;
    e = cudaFuncGetAttributes(&fa, noalloc_conserved_kernel<float>);
    if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, noalloc_conserved_kernel<double>);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = (NoallocScratch*)p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace lbm

extern "C" int lbm_conserved_noalloc(const void* f, int32_t precision, int32_t nx, int32_t ny, int32_t nz,
                                     const lbm_vset* vset, double* out, int32_t out_on_device, void* cuda_stream) {
  using namespace lbm;
  if (!f || !out || !vset) return LBM_EINVAL;
  if (precision != LBM_FP64 && precision != LBM_FP32) return LBM_EINVAL;
  if (nx < 1 || ny < 1 || nz < 1) return LBM_EINVAL;
  const long long n = (long long)nx * ny * nz;
  if (n > kNoallocMaxCells) return LBM_EINVAL;  // the static scratch holds 4096 block partials
  if (!(vset->c1 > 0) || !(vset->c2 > 0) || !(vset->eta0 > 0)) return LBM_EINVAL;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  // also makes the device's primary context current for the lookup below
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return LBM_ECUDA;
  if (cap != cudaStreamCaptureStatusNone && !out_on_device) return LBM_EINVAL;  // cannot synchronise
  NoallocScratch* scr = nullptr;
  if (scratch_for_current_device(&scr) != cudaSuccess) return LBM_ECUDA;
  Consts m;
  m.c1 = vset->c1;
  m.s = vset->c2 / std::sqrt(3.0);
  m.eta0sq = vset->eta0 * vset->eta0;
  m.c1sq = vset->c1 * vset->c1;
  m.c2sq = vset->c2 * vset->c2;
  if (cudaMemsetAsync(&scr->counter, 0, sizeof(unsigned), st) != cudaSuccess) return LBM_ECUDA;
  const int blocks = (int)((n + kNoallocCellsPerBlock - 1) / kNoallocCellsPerBlock);
  double* dst = out_on_device ? out : scr->result;
  if (precision == LBM_FP64)
    noalloc_conserved_kernel<double><<<blocks, kNoallocThreads, 0, st>>>((const double*)f, n, m, scr, dst);
  else
    noalloc_conserved_kernel<float><<<blocks, kNoallocThreads, 0, st>>>((const float*)f, n, m, scr, dst);
  if (cudaGetLastError() != cudaSuccess) return LBM_ECUDA;
  if (!out_on_device) {
    if (cudaMemcpyAsync(out, scr->result, 5 * sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
      return LBM_ECUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return LBM_ECUDA;
  }
  return LBM_OK;
}
