// 1-D CNN of the learned period proposal (sm_103a): the 64 -> 64 channel
// convolutions (kernel 9, "same" padding) as implicit GEMMs on the 5th-generation
// tensor cores, BF16 operands, FP32 accumulation in tensor memory.
//
// Layouts. Activations are channels-last BF16 [B][L][64] (one 128-byte row per
// position). A CTA computes a tile of 128 positions x 64 output channels:
//   Y[l, co] = sum_{kk=0..8} sum_{ci} W[kk][co][ci] X[l + kk - 4, ci]
// The 136 input rows l0-4 .. l0+131 are staged once per tile in shared memory in
// the no-swizzle K-major canonical layout, one "plane" per 8 input channels
// (rows at a 16-byte stride), so tap kk is the same tile shifted by kk rows: its
// A descriptor starts kk * 16 bytes later. The weights (9 taps x 64 x 64) stay
// resident in the same layout. One thread issues 9 taps x 4 K-steps of
// tcgen05.mma (M = 128, N = 64, K = 16); the accumulator (128 lanes x 64 FP32
// columns of TMEM) is read back with tcgen05.ld for the epilogue (bias, ReLU or
// the backward ReLU mask, BF16 store). Tiles are double-buffered: the next
// tile's rows are copied (cp.async, zero-filled outside [0, L)) while the MMAs
// of the current one run.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "qlp_internal.h"
#include "tc_common.cuh"

namespace qlp {

constexpr int kC = 64;             // channels of the middle layers
constexpr int kTaps = 9;           // kernel size
constexpr int kTileM = 128;        // positions per tile
constexpr int kRows = kTileM + kTaps - 1;  // staged rows per tile
constexpr int kPlanes = kC / 8;    // 8 channels (16 bytes) per plane
constexpr int kPlaneBytes = kRows * 16;    // 2,176
constexpr int kABytes = kPlanes * kPlaneBytes;  // 17,408
constexpr int kWBytes = kTaps * kPlanes * kC * 16;  // 73,728
constexpr uint32_t kWaitLimit = 1u << 26;

struct ConvTcArgs {
  const __nv_bfloat16* x;      // [B][L][64]
  const uint4* wpack;          // packed weights, kWBytes
  const float* bias;           // [64] or null
  const __nv_bfloat16* mask;   // [B][L][64]: multiply by (mask > 0) (backward), or null
  __nv_bfloat16* y;            // [B][L][64]
  int32_t* err;
  int32_t batch;
  int32_t len;                 // multiple of 128
  int32_t relu;
};

__device__ __forceinline__ void stage_tile(unsigned char* abuf, const __nv_bfloat16* x, int b, int l0,
                                           int len) {
  // plane j, row r  <-  x[b][l0 - 4 + r][8j .. 8j+7]
  for (int i = threadIdx.x; i < kPlanes * kRows; i += blockDim.x) {
    const int j = i / kRows, r = i - j * kRows;
    const int l = l0 - (kTaps / 2) + r;
    const bool in = l >= 0 && l < len;
    const __nv_bfloat16* src = x + ((size_t)b * len + (in ? l : 0)) * kC + 8 * j;
    cp_async16(abuf + j * kPlaneBytes + r * 16, src, in ? 16u : 0u);
  }
}

__global__ void __launch_bounds__(128) conv64_tc_kernel(const ConvTcArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* wsm = smem;
  unsigned char* abuf0 = smem + kWBytes;
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_per_sample = a.len / kTileM;
  const int n_tiles = a.batch * tiles_per_sample;

  // resident weights
  const uint4* wsrc = a.wpack;
  uint4* wdst = reinterpret_cast<uint4*>(wsm);
  for (int i = tid; i < kWBytes / 16; i += blockDim.x) wdst[i] = wsrc[i];
  if (tid == 0) {
    mbar_init(&mbar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    s_fail = 0;
  }
  if (warp == 0) tmem_alloc(&tmem_base, 64);
  int t = blockIdx.x;
  if (t < n_tiles) stage_tile(abuf0, a.x, t / tiles_per_sample, (t % tiles_per_sample) * kTileM, a.len);
  asm volatile("cp.async.commit_group;" ::: "memory");
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  const uint32_t idesc = idesc_bf16_f32(kTileM, kC);
  uint32_t phase = 0;
  int buf = 0;

  for (; t < n_tiles; t += gridDim.x) {
    const int b = t / tiles_per_sample;
    const int l0 = (t % tiles_per_sample) * kTileM;
    unsigned char* acur = abuf0 + buf * kABytes;
    cp_async_wait_all();
    fence_proxy_async_smem();  // the copies become visible to the tensor core
    __syncthreads();
    // prefetch the next tile into the other buffer
    const int tn = t + gridDim.x;
    if (tn < n_tiles)
      stage_tile(abuf0 + (buf ^ 1) * kABytes, a.x, tn / tiles_per_sample, (tn % tiles_per_sample) * kTileM,
                 a.len);
    asm volatile("cp.async.commit_group;" ::: "memory");

    if (tid == 0) {
      tc_fence_after();
      const uint32_t abase = smem_u32(acur), wbase = smem_u32(wsm);
      bool acc = false;
#pragma unroll 1
      for (int kk = 0; kk < kTaps; ++kk) {
#pragma unroll
        for (int ks = 0; ks < kPlanes / 2; ++ks) {
          const uint64_t ad = smem_desc(abase + 2 * ks * kPlaneBytes + kk * 16, kPlaneBytes, 128);
          const uint64_t bd = smem_desc(wbase + (kk * kPlanes + 2 * ks) * (kC * 16), kC * 16, 128);
          mma_bf16(tmem, ad, bd, idesc, acc);
          acc = true;
        }
      }
      mma_commit(&mbar);
    }
    const bool ok = mbar_wait(&mbar, phase, kWaitLimit);
    phase ^= 1;
    if (!ok) {
      if (lane == 0) atomicOr(a.err, kErrMmaWait);
      s_fail = 1;
    }
    tc_fence_after();
    // epilogue: row = 32 warp + lane, 64 columns
    const int row = 32 * warp + lane;
    const int l = l0 + row;
    __nv_bfloat16* yrow = a.y + ((size_t)b * a.len + l) * kC;
    const __nv_bfloat16* mrow = a.mask ? a.mask + ((size_t)b * a.len + l) * kC : nullptr;
#pragma unroll
    for (int c0 = 0; c0 < kC; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0, v);
      __align__(16) __nv_bfloat16 o[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        float z = v[i];
        if (a.bias) z += a.bias[c0 + i];
        if (a.relu) z = fmaxf(z, 0.f);
        if (mrow) z = (__bfloat162float(mrow[c0 + i]) > 0.f) ? z : 0.f;
        o[i] = __float2bfloat16_rn(z);
      }
      uint4* dst = reinterpret_cast<uint4*>(yrow + c0);
      dst[0] = reinterpret_cast<const uint4*>(o)[0];
      dst[1] = reinterpret_cast<const uint4*>(o)[1];
    }
    tc_fence_before();
    __syncthreads();
    if (s_fail) break;
    buf ^= 1;
  }
  cp_async_wait_all();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 64);
}

// W[kk][co][ci] (FP32) -> BF16 planes for the tensor-core kernel. transpose=1
// packs the weights of the input-gradient convolution: W'[kk][ci][co] = W[8-kk][co][ci].
__global__ void pack_w64_kernel(const float* w, uint4* out, int transpose) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (kk, plane j, row n)
  if (i >= kTaps * kPlanes * kC) return;
  const int kk = i / (kPlanes * kC);
  const int j = (i / kC) % kPlanes;
  const int n = i % kC;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = 8 * j + e;  // reduction channel
    const float x = transpose ? w[((kTaps - 1 - kk) * kC + k) * kC + n] : w[(kk * kC + n) * kC + k];
    v[e] = __float2bfloat16_rn(x);
  }
  out[i] = *reinterpret_cast<const uint4*>(v);
}

// Shared memory of the conv kernel: resident weights and two row tiles.
int conv64_smem_bytes() { return kWBytes + 2 * kABytes; }

int launch_conv64(const void* xv, const void* wv, const float* bias, const void* mv, void* yv,
                  int32_t* err, int batch, int len, int relu, void* stream) {
  const __nv_bfloat16* x = static_cast<const __nv_bfloat16*>(xv);
  const uint4* wpack = static_cast<const uint4*>(wv);
  const __nv_bfloat16* mask = static_cast<const __nv_bfloat16*>(mv);
  __nv_bfloat16* y = static_cast<__nv_bfloat16*>(yv);
  if (batch <= 0) return 0;
  const int smem = conv64_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(conv64_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = batch * (len / kTileM);
  const int grid = tiles < 2 * sms ? tiles : 2 * sms;
  ConvTcArgs a{x, wpack, bias, mask, y, err, batch, len, relu};
  conv64_tc_kernel<<<grid, 128, smem, (cudaStream_t)stream>>>(a);
  return (int)cudaGetLastError();
}

int launch_pack_w64(const float* w, void* out, int transpose, void* stream) {
  const int n = kTaps * kPlanes * kC;
  pack_w64_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(w, static_cast<uint4*>(out), transpose);
  return (int)cudaGetLastError();
}

}  // namespace qlp
