// mm_gram_tma.cu -- stage (d) for many assets: the covariance of Algorithm 3
// step C (Eqs. (2)/(3)) as Sigma = A A^T on the tensor cores with the split
// operand prepared once and streamed by the Tensor Memory Accelerator.
//
// A is the real D x 2(N+1) matrix whose row i holds s_k Re F_i(k), s_k Im
// F_i(k) (k = 0..N, s_k = 2 pi sqrt(W_k), W_0 = w_0, W_k = 2 w_k; see
// mm_gram.cu). Where the contraction is tensor-bound, converting A to split
// precision inside it (about two dozen instructions per complex value, by
// every CTA that reads the tile) costs more issue slots than the MMAs it
// feeds. Here a streaming pass writes A once as hi and lo planes (bf16 for
// BF16x3, tf32 in float32 containers for 3xTF32), row-major with rows padded
// to whole K-chunks of 128 bytes and the row count padded to whole 128-row
// tiles (pad rows stay zero). The contraction then runs three roles per CTA
// (one output tile pair I <= J and one range of K-chunks):
//  * a producer thread issues cp.async.bulk.tensor loads of the chunk's hi
//    and lo tiles of rows I (and J) into a ring of shared-memory stages,
//    128-byte swizzled by the tensor map so that they land in the canonical
//    K-major layout of the MMA descriptors;
//  * an MMA thread waits for each stage, issues hi*hi + hi*lo + lo*hi into a
//    TMEM accumulator and commits the stage back to the producer;
//  * four epilogue warps wait for the last commit, read TMEM (one lane
//    quadrant each) and add the partial tile into the FP32 accumulator with
//    vector reductions in L2, as the other tensor-core path does.
// Every wait is bounded by the plan's limit; a CTA that gives up waits (at
// the fixed limit) for its own copies and MMAs in flight, records
// ST_TIMEOUT, frees its TMEM and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <mutex>

#include "mm_async.cuh"
#include "mm_common.cuh"
#include "mm_tc.cuh"

namespace mmgpu {

// ------------------------------------------------------------ split pass
// Row a of the operand: complex mode k -> elements 2k, 2k+1 of both planes;
// modes N < k < kpc are zero. Each thread takes four consecutive modes: four
// 8-byte coefficient loads in flight and one 16-byte store per plane (bf16)
// or two (tf32); kpc is a multiple of 16, so a row's quads never straddle.
constexpr int kSplitModes = 4;

template <int MODE>
__global__ void __launch_bounds__(256) k_gram_split(const float2* __restrict__ F, GramParams g,
                                                    const float* __restrict__ wsq, void* __restrict__ hi,
                                                    void* __restrict__ lo, int kpc) {
  pdl_wait();  // the coefficients come from the FFT kernel
  pdl_trigger();
  const int a = blockIdx.y;
  const int k0 = (blockIdx.x * blockDim.x + threadIdx.x) * kSplitModes;
  if (k0 >= kpc) return;
  float xr[kSplitModes], xi[kSplitModes];
  const float2* row = F + (int64_t)a * g.ld;
#pragma unroll
  for (int q = 0; q < kSplitModes; ++q) {
    const int k = k0 + q;
    xr[q] = 0.f;
    xi[q] = 0.f;
    if (k <= g.N) {
      const float sc = __ldg(wsq + k);
      const float2 f = __ldg(row + k);
      xr[q] = f.x * sc;
      xi[q] = f.y * sc;
    }
  }
  const int64_t o = (int64_t)a * kpc + k0;  // in complex modes
  if (MODE == 0) {
    uint32_t h[kSplitModes], l[kSplitModes];
#pragma unroll
    for (int q = 0; q < kSplitModes; ++q) {
      const __nv_bfloat162 H = __floats2bfloat162_rn(xr[q], xi[q]);
      const __nv_bfloat162 L = __floats2bfloat162_rn(xr[q] - __low2float(H), xi[q] - __high2float(H));
      h[q] = *reinterpret_cast<const uint32_t*>(&H);
      l[q] = *reinterpret_cast<const uint32_t*>(&L);
    }
    reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(hi) + o)[0] = make_uint4(h[0], h[1], h[2], h[3]);
    reinterpret_cast<uint4*>(reinterpret_cast<uint32_t*>(lo) + o)[0] = make_uint4(l[0], l[1], l[2], l[3]);
  } else {
    uint32_t h[2 * kSplitModes], l[2 * kSplitModes];
#pragma unroll
    for (int q = 0; q < kSplitModes; ++q) {
      h[2 * q] = f32_to_tf32(xr[q]);
      h[2 * q + 1] = f32_to_tf32(xi[q]);
      l[2 * q] = f32_to_tf32(xr[q] - __uint_as_float(h[2 * q]));
      l[2 * q + 1] = f32_to_tf32(xi[q] - __uint_as_float(h[2 * q + 1]));
    }
    uint4* hp = reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(hi) + o);
    uint4* lp = reinterpret_cast<uint4*>(reinterpret_cast<uint2*>(lo) + o);
    hp[0] = make_uint4(h[0], h[1], h[2], h[3]);
    hp[1] = make_uint4(h[4], h[5], h[6], h[7]);
    lp[0] = make_uint4(l[0], l[1], l[2], l[3]);
    lp[1] = make_uint4(l[4], l[5], l[6], l[7]);
  }
}

// ------------------------------------------------------------ contraction
constexpr int kTmaThreads = 192;  // warp 0 producer + TMEM, warp 1 MMA, warps 2-5 epilogue
constexpr int kTmaMaxStages = 8;
constexpr size_t kTmaStageBudget = 196608;  // bytes of stages per CTA (one CTA per SM)

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <int MODE>
__global__ void __launch_bounds__(kTmaThreads, 1) k_gram_tma(const __grid_constant__ CUtensorMap map_hi,
                                                             const __grid_constant__ CUtensorMap map_lo, GramParams g,
                                                             float* __restrict__ acc, int* status, int nst) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  __shared__ __align__(8) uint64_t full[kTmaMaxStages], empty[kTmaMaxStages], done;
  __shared__ uint32_t s_tmem;
  __shared__ int s_fail;

  int I, J;
  pair_of(blockIdx.y, g.ntiles, I, J);
  const bool two = I != J;
  const int s = blockIdx.x;
  const int c0 = (int)((int64_t)s * g.nchunks / g.splits);
  const int c1 = (int)((int64_t)(s + 1) * g.nchunks / g.splits);
  const int nit = c1 - c0;
  const uint32_t base_s = smem_u32(smem_raw);
  uint8_t* base = smem_raw + (((base_s + 1023u) & ~1023u) - base_s);
  const uint32_t stage_bytes = (two ? 4u : 2u) * (uint32_t)kTileBytes;
  const int rowsI = min(kTile, g.D - I * kTile);
  const int rowsJ = min(kTile, g.D - J * kTile);
  const int Nmma = ((rowsJ + 15) / 16) * 16;
  const uint32_t fmt = (MODE == 0) ? 1u : 2u;  // bf16 / tf32 operands
  const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(Nmma >> 3) << 17) |
                         ((uint32_t)(kTile >> 4) << 24);
  constexpr int kChunkElems = MODE == 0 ? 64 : 32;  // 128 bytes of one operand row
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int i = 0; i < nst; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(&done, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_hi)) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_lo)) : "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = s_tmem;
  pdl_wait();     // the operand planes come from the split pass
  pdl_trigger();  // the correlation epilogue may be scheduled

  if (warp == 0 && lane == 0) {
    // producer: stage it % nst takes chunk c0 + it once the MMAs of chunk
    // it - nst have released it
    int issued = 0;
    for (int it = 0; it < nit; ++it) {
      const int st = it % nst;
      if (it >= nst && !mbar_wait(&empty[st], (uint32_t)(((it / nst) & 1) ^ 1), g.wait_ns)) {
        atomicOr(&s_fail, 1);
        break;
      }
      uint8_t* stg = base + (size_t)st * stage_bytes;
      mbar_expect_tx(&full[st], stage_bytes);
      const int x = (c0 + it) * kChunkElems;
      tma_load_2d(stg, &map_hi, x, I * kTile, &full[st]);
      tma_load_2d(stg + kTileBytes, &map_lo, x, I * kTile, &full[st]);
      if (two) {
        tma_load_2d(stg + 2 * kTileBytes, &map_hi, x, J * kTile, &full[st]);
        tma_load_2d(stg + 3 * kTileBytes, &map_lo, x, J * kTile, &full[st]);
      }
      issued = it + 1;
    }
    // no copy may still be landing when the CTA leaves
    for (int it = issued > nst ? issued - nst : 0; it < issued; ++it)
      mbar_wait(&full[it % nst], (uint32_t)((it / nst) & 1), kWaitLimitNs);
  } else if (warp == 1 && lane == 0) {
    // MMA issue
    for (int it = 0; it < nit; ++it) {
      const int st = it % nst;
      if (!mbar_wait(&full[st], (uint32_t)((it / nst) & 1), g.wait_ns)) {
        atomicOr(&s_fail, 1);
        break;
      }
      tc_fence_after();
      const uint32_t a_hi = smem_u32(base + (size_t)st * stage_bytes), a_lo = a_hi + kTileBytes;
      const uint32_t b_hi = two ? a_hi + 2 * kTileBytes : a_hi;
      const uint32_t b_lo = two ? a_hi + 3 * kTileBytes : a_lo;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {  // four 32-byte K steps per 128-byte row
        const uint32_t o = ks * 32;
        tc_mma<MODE>(tmem, sw128_desc(a_hi + o), sw128_desc(b_hi + o), idesc, (it > 0 || ks > 0) ? 1u : 0u);
        tc_mma<MODE>(tmem, sw128_desc(a_hi + o), sw128_desc(b_lo + o), idesc, 1u);
        tc_mma<MODE>(tmem, sw128_desc(a_lo + o), sw128_desc(b_hi + o), idesc, 1u);
      }
      tc_commit(&empty[st]);  // the stage is free once these MMAs have read it
    }
    tc_commit(&done);  // completes when every MMA issued above has
  } else if (warp >= 2) {
    if (!mbar_wait(&done, 0, g.wait_ns)) {
      atomicOr(&s_fail, 1);
      mbar_wait(&done, 0, kWaitLimitNs);  // the issued MMAs still finish before TMEM is read or freed
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (!s_fail && nit > 0) {
    if (warp >= 2) {
      // warp w reads TMEM lanes 32 (w mod 4) .. + 31 (its lane quadrant)
      const int quad = warp & 3;
      const int r = quad * 32 + lane;
      float* out = acc + (int64_t)(I * kTile + r) * g.Dp + J * kTile;
      for (int c = 0; c < Nmma; c += 16) {
        uint32_t v[16];
        tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c, v);
        if (r < rowsI) {
#pragma unroll
          for (int q = 0; q < 4; ++q)
            if (c + 4 * q < rowsJ)
              red_add_v4(out + c + 4 * q, __uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]),
                         __uint_as_float(v[4 * q + 2]), __uint_as_float(v[4 * q + 3]));
        }
      }
    }
  } else if (s_fail && threadIdx.x == 0) {
    atomicOr(status, ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

// ------------------------------------------------------------ host side
namespace {

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::once_flag g_encode_once;

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  std::call_once(g_encode_once, [] {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q{};
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  });
  return g_encode;
}

// 2-D map over one operand plane: rows of kpc complex modes (2 kpc
// elements), Dpad rows; boxes of 128 bytes x 128 rows, 128-byte swizzle.
bool encode_plane(CUtensorMap* map, int mode, void* plane, int kpc, int Dpad) {
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (!enc) return false;
  const size_t es = mode == 0 ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)2 * kpc, (cuuint64_t)Dpad};
  const cuuint64_t strides[1] = {(cuuint64_t)2 * kpc * es};
  const cuuint32_t box[2] = {(cuuint32_t)(128 / es), (cuuint32_t)kTile};
  const cuuint32_t estr[2] = {1, 1};
  const CUresult r =
      enc(map, mode == 0 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, plane, dims,
          strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
          CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace

int gram_tma_kpc(const GramParams& g) { return g.chunk * g.nchunks; }

size_t gram_tma_plane_bytes(int mode, int D, int N_max, int chunk) {
  const size_t kpc = (size_t)chunk * ((N_max + 1 + chunk - 1) / chunk);
  const size_t Dpad = ((size_t)D + kTile - 1) / kTile * kTile;
  return Dpad * kpc * 2 * (mode == 0 ? 2 : 4);
}

cudaError_t launch_gram_split(int mode, const void* coeffs, const GramParams& g, const float* wsq, void* hi, void* lo,
                              cudaStream_t s) {
  const int kpc = gram_tma_kpc(g);
  dim3 grd((kpc / kSplitModes + 255) / 256, g.D);
  if (mode == 0)
    return launch_pdl(k_gram_split<0>, grd, dim3(256), 0, s, (const float2*)coeffs, g, wsq, hi, lo, kpc);
  return launch_pdl(k_gram_split<1>, grd, dim3(256), 0, s, (const float2*)coeffs, g, wsq, hi, lo, kpc);
}

cudaError_t launch_gram_tma(int mode, const GramParams& g, void* hi, void* lo, float* acc, int* status,
                            cudaStream_t s) {
  const int kpc = gram_tma_kpc(g);
  const int Dpad = g.ntiles * kTile;
  CUtensorMap mh, ml;
  if (!encode_plane(&mh, mode, hi, kpc, Dpad) || !encode_plane(&ml, mode, lo, kpc, Dpad))
    return cudaErrorInvalidValue;
  const bool two = g.ntiles > 1;
  const size_t stage = (size_t)(two ? 4 : 2) * kTileBytes;
  const int nst = (int)std::min<size_t>(kTmaMaxStages, kTmaStageBudget / stage);
  const size_t smem = (size_t)nst * stage + 1024;  // + alignment slack
  dim3 grd(g.splits, g.npairs);
  cudaError_t e;
  if (mode == 0) {
    e = cudaFuncSetAttribute(k_gram_tma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    return launch_pdl(k_gram_tma<0>, grd, dim3(kTmaThreads), smem, s, mh, ml, g, acc, status, nst);
  }
  e = cudaFuncSetAttribute(k_gram_tma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_gram_tma<1>, grd, dim3(kTmaThreads), smem, s, mh, ml, g, acc, status, nst);
}

}  // namespace mmgpu
