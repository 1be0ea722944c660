// Allocation-free residual norms (biot_residual_norms_noalloc).
//
// Callers that own all device memory through their own pool or arena cannot let
// a library call cudaMalloc/cudaFree (those calls synchronise the device and
// fragment the caller's pool). This entry point computes the same window
// residual and relative norms as biot_residual_norms from device buffers the
// caller passes in; the only scratch it needs -- per-block partial sums of the
// two norms -- lives in the file-scope device array below, whose device address
// is looked up once per device with cudaGetSymbolAddress. Nothing is allocated.
#include "common.cuh"

#include <cmath>
#include <mutex>

namespace biot {
namespace {

constexpr int kNoAllocMaxCols = BIOT_NOALLOC_MAX_COLS;
constexpr int kMaxDevices = 128;

// Partial sums [slot 0: |D^{-1/2} r|^2, slot 1: |D^{-1/2} b|^2][kRedBlocks][kNoAllocMaxCols]:
// 2 x 304 x 512 doubles = 2.49 MB on every device that loads the library, until exit.
// Every call overwrites each partial it reads, so nothing has to start at zero.
static __device__ __align__(256) double g_noalloc_partials[2 * kRedBlocks * kNoAllocMaxCols];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

// rel[c] = |D^{-1/2} r_c| / |D^{-1/2} b_c|; the blocks are summed in order, as
// the context path's two-level reduction does.
__global__ void k_rel_from_partials(const double* __restrict__ part, int nblocks, int ldp, int ncols,
                                    double* __restrict__ rel) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncols) return;
  double rr = 0.0, bb = 0.0;
  for (int b = 0; b < nblocks; ++b) rr += part[(size_t)b * ldp + c];
  for (int b = 0; b < nblocks; ++b) bb += part[(size_t)(nblocks + b) * ldp + c];
  const double r = sqrt(rr), q = sqrt(bb);
  rel[c] = q > 0.0 ? r / q : (r == 0.0 ? 0.0 : INFINITY);
}

// Device address of g_noalloc_partials on the current device. Looked up on the first call
// per device; looked up again on every call whose stream is not capturing, so that a
// device reset (which reloads the module at a possibly different address) is followed.
// A capturing stream uses the address cached by an earlier call.
biot_status scratch_address(cudaStream_t s, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(nullptr, BIOT_E_CUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return fail(nullptr, BIOT_E_CUDA, "device ordinal %d unsupported", dev);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(s, &cap);
  if (e != cudaSuccess) return fail(nullptr, BIOT_E_CUDA, "cudaStreamIsCapturing: %s", cudaGetErrorString(e));
  std::lock_guard<std::mutex> lock(g_addr_mu);
  if (!g_addr[dev] || cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || p == nullptr)
      return fail(nullptr, BIOT_E_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return BIOT_OK;
}

}  // namespace
}  // namespace biot

using namespace biot;

extern "C" biot_status biot_residual_norms_noalloc(int32_t n_nodes, const int32_t* nodeptr, const int32_t* nbr,
                                                   const int32_t* rowptr, const double* val, const double* ap_pp,
                                                   const double* dscale, const double* X, const double* F,
                                                   int32_t ldx, int32_t lo, int32_t ncols, double* R, int32_t ldr,
                                                   double* rel, void* cuda_stream) {
  if (!nodeptr || !nbr || !rowptr || !val || !ap_pp || !dscale || !X || !F || !R || !rel)
    return fail(nullptr, BIOT_E_INVALID, "biot_residual_norms_noalloc: NULL buffer");
  if (n_nodes < 1) return fail(nullptr, BIOT_E_INVALID, "biot_residual_norms_noalloc: n_nodes must be >= 1");
  if (ncols < 1 || ncols > kNoAllocMaxCols)
    return fail(nullptr, BIOT_E_INVALID, "biot_residual_norms_noalloc: ncols = %d outside 1..%d (fixed scratch size)",
                ncols, kNoAllocMaxCols);
  // in 64 bits: lo + ncols overflows int32 for lo near INT32_MAX
  if (lo < 1 || (int64_t)ldx < (int64_t)lo + ncols || ldr < ncols)
    return fail(nullptr, BIOT_E_INVALID, "biot_residual_norms_noalloc: need lo >= 1, ldx >= lo + ncols, ldr >= ncols");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  void* part = nullptr;
  BIOT_TRY(scratch_address(s, &part));
  double* p = static_cast<double*>(part);
  launch_residual_raw(n_nodes, nodeptr, nbr, rowptr, val, ap_pp, dscale, X, F, ldx, lo, ncols, R, ldr, p,
                      kNoAllocMaxCols, s);
  BIOT_LAUNCH(k_rel_from_partials, div_up(ncols, 128), 128, 0, s, p, kRedBlocks, kNoAllocMaxCols, ncols, rel);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(nullptr, BIOT_E_CUDA, "biot_residual_norms_noalloc launch: %s", cudaGetErrorString(e));
  return BIOT_OK;
}
