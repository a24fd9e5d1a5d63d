// Allocation-free variant of the small-exponential entry point (etp_expm_e1).
//
// Some callers cannot allocate device memory: real-time loops in which
// cudaMalloc could stall or synchronise the device, processes that fix their
// device-memory budget at start-up, or hosts whose device memory belongs to
// another allocator that hands out fixed buffers. etp_expm_e1_noalloc takes
// device pointers for its input and output and keeps its workspace in one
// file-scope static device array instead of calling cudaMalloc.
#include <mutex>

#include "etp_host.cuh"
#include "expm_kernels.cuh"

namespace etp {

constexpr int kNoAllocMaxN = 64;
// six n x n workspace matrices (B, B^2, B^3, B^4, R0, R1) plus the scaling exponent
constexpr size_t kNoAllocDoubles = (size_t)EXPM_NMAT * kNoAllocMaxN * kNoAllocMaxN + 32;

// Held by every GPU that loads the library, until the process exits (~192 KiB).
static __device__ __align__(256) double g_expm_scratch[kNoAllocDoubles];

constexpr int kMaxDevices = 64;
static double* g_scratch_addr[kMaxDevices] = {};
static std::mutex g_scratch_mutex;

// Device address of the static scratch on `device` (which must be current).
// Looked up once per device: host code may not use the symbol itself, which is
// only a host-side stand-in for the device array.
static etp_status scratch_for_device(int device, double** out) {
  if (device < 0 || device >= kMaxDevices) return fail(ETP_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_expm_scratch);
    if (e != cudaSuccess || !p)
      return fail(ETP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_scratch_addr[device] = (double*)p;
  }
  *out = g_scratch_addr[device];
  return ETP_OK;
}

}  // namespace etp

using namespace etp;

extern "C" etp_status etp_expm_e1_noalloc(etp_ctx* ctx, int n, const double* H, double tau, double* y) {
  if (!ctx || !H || !y) return fail(ETP_ERR_INVALID, "null argument");
  if (n < 1 || n > kNoAllocMaxN)
    return fail(ETP_ERR_INVALID, "etp_expm_e1_noalloc: n must be in 1..64 (the size its static scratch holds)");
  ETP_CUDA_TRY(cudaSetDevice(ctx->device));
  double* scratch = nullptr;
  ETP_TRY(scratch_for_device(ctx->device, &scratch));
  cudaStream_t st = ctx->stream;
  ExpmParams p{};
  p.H = H;
  p.ldH = n;
  p.j0 = n;
  p.ncand = 1;
  p.tau = tau;
  p.ws = scratch;  // every workspace entry a call reads is written earlier in that call
  p.ld = n;
  p.s_arr = (int*)(scratch + (size_t)EXPM_NMAT * n * n);
  p.ks = nullptr;
  double f = 1.0;
  for (int k = 0; k <= EXPM_TAYLOR_DEG; ++k) {
    if (k > 1) f *= k;
    p.coef[k] = 1.0 / f;
  }
  const unsigned gx = (unsigned)((n * n + 63) / 64);
  k_expm_prep<<<1, 256, 0, st>>>(p);
  k_expm_mm<<<dim3(gx, 1, 1), 64, 0, st>>>(p, 0, 0);
  k_expm_mm<<<dim3(gx, 1, 2), 64, 0, st>>>(p, 1, 0);
  for (int k = 3; k >= 0; --k) k_expm_mm<<<dim3(gx, 1, 1), 64, 0, st>>>(p, 2, k);
  ETP_CUDA_TRY(cudaGetLastError());
  int s = 0;  // scaling exponent, read back to launch exactly s squarings
  ETP_CUDA_TRY(cudaMemcpyAsync(&s, p.s_arr, sizeof(int), cudaMemcpyDeviceToHost, st));
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  for (int k = 0; k < s; ++k) k_expm_mm<<<dim3(gx, 1, 1), 64, 0, st>>>(p, 3, k);
  k_expm_first_column<<<1, 128, 0, st>>>(p, y);
  ETP_CUDA_TRY(cudaGetLastError());
  ETP_CUDA_TRY(cudaStreamSynchronize(st));
  ctx->launches += 8 + s;
  return ETP_OK;
}
