// mm_noalloc.cu -- mm_corr_noalloc: the covariance / correlation contraction
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code running where the allocator is
// owned by someone else (a memory pool that must not grow, a host process
// whose allocations are audited), or where an allocation could fail at a bad
// time. For them this entry point runs the same split-K contraction kernels
// as mm_corr without a plan, taking its scratch (the basis weights, the
// split-K partial tiles and a status word) from one file-scope device array.
//
// Limits: 1 <= D <= 128, 0 <= N <= 65535, at most 16 K-splits (the FP64
// path's partial tiles; the mixed path uses the same bytes as its 128 x 128
// float accumulator). The array is
// about 2 MB and every GPU that loads the library holds it until the process
// exits. Every call shares it, so calls that overlap on the GPU (different
// streams, or host threads without ordering) race and give wrong results.
#include <mutex>

#include "mm_common.cuh"

using namespace mmgpu;

namespace {

constexpr int kNaMaxD = 128;
constexpr int kNaMaxN = 65535;
constexpr int kNaMaxSplits = 16;
// partial tiles: FP32 path 1 pair of 128 x 128 floats; FP64 path up to
// 3 pairs of 64 x 64 doubles (D <= 128 gives at most 2 x 2 tiles of 64)
constexpr size_t kNaPartialBytes = (size_t)kNaMaxSplits * 3 * 64 * 64 * 8;  // >= the FP32 accumulator
constexpr size_t kNaWeightBytes = (size_t)(kNaMaxN + 1) * 8;
constexpr size_t kNaStatusBytes = 256;
constexpr size_t kNaBytes = kNaPartialBytes + kNaWeightBytes + kNaStatusBytes;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaBytes];

constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
void* g_na_base[kNaMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (host code cannot use the array's name as a device address).
mm_status scratch_base(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return MM_ERR_CUDA;
  std::lock_guard<std::mutex> lk(g_na_mutex);
  if (!g_na_base[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MM_ERR_CUDA;
    }
    g_na_base[dev] = p;
  }
  *out = g_na_base[dev];
  return MM_OK;
}

mm_status map_flags(int f) {
  if (f & ST_TIMEOUT) return MM_ERR_TIMEOUT;
  if (f & ST_ZERO_VAR) return MM_ERR_ZERO_VARIANCE;
  return MM_OK;
}

}  // namespace

extern "C" mm_status mm_corr_noalloc(int32_t D, int32_t N, mm_basis basis, mm_precision prec,
                                     const void* d_coeffs, void* d_sigma_or_null, void* d_R, void* stream) {
  if (!d_coeffs || !d_R) return MM_ERR_INVALID_ARG;
  if (basis != MM_BASIS_DIRICHLET && basis != MM_BASIS_FEJER) return MM_ERR_INVALID_ARG;
  if (prec < MM_PREC_FP64 || prec > MM_PREC_MIXED_3XTF32) return MM_ERR_INVALID_ARG;
  if (D < 1 || N < 0) return MM_ERR_INVALID_ARG;
  if (D > kNaMaxD || N > kNaMaxN) return MM_ERR_UNSUPPORTED;  // beyond the fixed scratch
  if (basis == MM_BASIS_FEJER && N < 1) return MM_ERR_CUTOFF;
  // the call reads its status back and synchronises the stream, which a
  // stream being captured into a graph does not allow
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing((cudaStream_t)stream, &cap) != cudaSuccess) {
    cudaGetLastError();
    return MM_ERR_INVALID_ARG;
  }
  if (cap != cudaStreamCaptureStatusNone) return MM_ERR_INVALID_ARG;
  void* base = nullptr;
  mm_status r = scratch_base(&base);
  if (r != MM_OK) return r;
  unsigned char* b = static_cast<unsigned char*>(base);
  void* partial = b;
  void* wsq = b + kNaPartialBytes;
  int* status = reinterpret_cast<int*>(b + kNaPartialBytes + kNaWeightBytes);

  const bool fp64 = prec == MM_PREC_FP64;
  GramParams g{};
  g.wait_ns = kDefaultWaitNs;
  g.D = D;
  g.N = N;
  g.ld = N + 1;
  g.Dp = (D + 3) / 4 * 4;
  g.tile = fp64 ? 64 : 128;
  g.ntiles = (D + g.tile - 1) / g.tile;
  g.npairs = g.ntiles * (g.ntiles + 1) / 2;
  g.chunk = fp64 ? 16 : (prec == MM_PREC_MIXED_BF16X3 ? 32 : 16);
  g.nchunks = (N + 1 + g.chunk - 1) / g.chunk;
  const int S = g.nchunks < kNaMaxSplits ? g.nchunks : kNaMaxSplits;
  g.chunks_per_split = (g.nchunks + S - 1) / S;
  g.splits = (g.nchunks + g.chunks_per_split - 1) / g.chunks_per_split;

  cudaStream_t st = (cudaStream_t)stream;
  // the status word and the mixed path's accumulator must start at zero; the
  // FP64 partial tiles and the weights are fully rewritten by the kernels
  if (cudaMemsetAsync(status, 0, sizeof(int), st) != cudaSuccess) return MM_ERR_CUDA;
  if (launch_gram_weights(basis, N, fp64, wsq, st) != cudaSuccess) return MM_ERR_CUDA;
  if (fp64) {
    if (launch_gram_f64(d_coeffs, g, (const double*)wsq, (double*)partial, st) != cudaSuccess) return MM_ERR_CUDA;
    if (launch_reduce_corr(true, partial, g, d_sigma_or_null, d_R, status, st) != cudaSuccess) return MM_ERR_CUDA;
  } else {
    float* acc = (float*)partial;
    if (cudaMemsetAsync(acc, 0, (size_t)D * g.Dp * sizeof(float), st) != cudaSuccess) return MM_ERR_CUDA;
    if (launch_gram_tc(prec == MM_PREC_MIXED_BF16X3 ? 0 : 1, d_coeffs, g, (const float*)wsq, acc, status, nullptr,
                       nullptr, nullptr, nullptr, st) != cudaSuccess)
      return MM_ERR_CUDA;
    if (launch_corr_acc(acc, g, (float*)d_sigma_or_null, (float*)d_R, nullptr, status, st) != cudaSuccess)
      return MM_ERR_CUDA;
  }
  int f = 0;
  if (cudaMemcpyAsync(&f, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess) return MM_ERR_CUDA;
  if (cudaStreamSynchronize(st) != cudaSuccess) return MM_ERR_CUDA;
  return map_flags(f);
}
