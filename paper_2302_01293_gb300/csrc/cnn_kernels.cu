// 1-D CNN of the learned period proposal (sm_103a): the 64 -> 64 channel
// convolutions (kernel 9, "same" padding) as implicit GEMMs on the 5th-generation
// tensor cores, BF16 operands, FP32 accumulation in tensor memory.
//
// Layouts. Activations are channels-last BF16 [B][L][64] (one 128-byte row per
// position). A tile is 128 positions x 64 output channels:
//   Y[l, co] = sum_{kk=0..8} sum_{ci} W[kk][co][ci] X[l + kk - 4, ci]
// Its 136 input rows l0-4 .. l0+131 sit in shared memory as they are in memory,
// one 128-byte row per position, in the 128-byte-swizzled K-major layout (chunk c
// of row r at chunk c ^ (r & 7)), so tap kk is the same tile shifted by kk rows:
// its A descriptor starts kk * 128 bytes later (the swizzle follows the address
// bits, so a shifted start reads the shifted rows). The weights (9 taps x 64 x 64)
// stay resident in the same layout, 64 rows of 128 bytes per tap. Each tile takes
// 9 taps x 4 K-steps of tcgen05.mma (M = 128, N = 64, K = 16, the K step 32 bytes
// along the row) into a TMEM accumulator of 64 FP32 columns.
//
// Pipeline (one persistent CTA per SM, warp roles): warp 0 copies the weights in
// one bulk asynchronous copy (on their own barrier, which the MMA issuer waits for)
// and loads tiles with TMA into a ring of kStages buffers (one box of 64 channels x 136 rows per tile, of a
// 3-D tensor map over [B][L][64] with the 128-byte swizzle, so rows outside
// [0, L) of the tile's own sample come back as zeros); warp 1 issues the MMAs of
// each tile into one of kAcc accumulators and commits them to the buffer's
// "empty" barrier and the accumulator's "full" barrier; warps 2-9 (two per TMEM
// lane quarter, 32 output channels each) read an accumulator back (one tcgen05.ld
// of 32 columns), apply bias and ReLU or the backward ReLU mask, store BF16 and
// release the accumulator. Every barrier wait
// is bounded; a wait that runs out raises QLP error bit 16, and the CTA still
// waits (bounded) for its copies and MMAs in flight before it frees TMEM.
#include <cuda.h>
#include <cudaTypedefs.h>
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
constexpr int kPlanes = kC / 8;    // 8 channels (16 bytes) per plane (the weight-gradient kernel's layout)
constexpr int kABytes = kRows * kC * 2;     // 17,408 = 17 swizzle atoms of 1,024 bytes
constexpr int kWBytes = kTaps * kC * kC * 2;  // 73,728 = 72 atoms
constexpr int kStages = 6;         // tile buffers in flight
constexpr int kAcc = 4;            // TMEM accumulators (64 columns each)
constexpr int kEpiWarps = 8;       // two per TMEM lane quarter, 32 columns each
constexpr int kConvThreads = 64 + 32 * kEpiWarps;  // producer, MMA, epilogue warps
constexpr int kOutBytes = kTileM * kC * 2;  // one BF16 output tile (16 KB), staged for a TMA store
constexpr int kOutBufs = 2;
constexpr uint32_t kWaitLimit = 1u << 26;

struct ConvTcArgs {
  const uint4* wpack;          // packed weights, kWBytes
  const float* bias;           // [64] or null
  const __nv_bfloat16* mask;   // [B][L][64]: multiply by (mask > 0) (backward), or null
  int32_t* err;
  int32_t batch;
  int32_t len;                 // multiple of 128
  int32_t relu;
};

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
// One TMA box of the 3-D map (channel x, row y, sample z) into shared memory,
// completing `bytes` on the barrier. x must be a multiple of 8 (16 bytes).
__device__ __forceinline__ void tma_load3(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// A shared-memory box to the 3-D map (channel x, row y, sample z) as one bulk group
// of this thread. x = 0 and y >= 0: the store starts at a 16-byte boundary.
__device__ __forceinline__ void tma_store3(const CUtensorMap* map, const void* src, int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%1, %2, %3}], [%4];\n\t"
      "cp.async.bulk.commit_group;" ::"l"(reinterpret_cast<uint64_t>(map)),
      "r"(x), "r"(y), "r"(z), "r"(smem_u32(src))
      : "memory");
}
// This thread's bulk groups have finished reading shared memory / have completed.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Barrier of the epilogue warps (id 1) that also ANDs a predicate over them.
__device__ __forceinline__ bool epi_barrier_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\t"
      "barrier.cta.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(32 * kEpiWarps)
      : "memory");
  return r != 0;
}

// Epilogue of one tile: accumulator columns [col + c0, col + c0 + 32) (output
// channels c0 .. c0+31) for the lane quarter q of this warp, row r = 32 q + lane;
// one TMEM load and wait, the accumulator released, then bias, ReLU or the backward
// mask, BF16, into the staging tile `out` (128 rows of 128 bytes, 1024-byte aligned)
// with the 128-byte swizzle of the store's tensor map: 16-byte chunk j of row r at
// chunk j ^ (r & 7), so that eight lanes fill the 32 banks once. The backward mask
// (the row's 32 channels, 4 chunks) was read by the caller before the accumulator wait.
__device__ __forceinline__ void conv_epilogue(const ConvTcArgs& a, const float* s_bias, uint32_t tmem,
                                              uint32_t col, int c0, int q, uint64_t* acc_empty,
                                              unsigned char* out, const uint4* mk) {
  const int lane = threadIdx.x & 31;
  const int r = 32 * q + lane;
  const bool mrow = a.mask != nullptr;
  float v[32];
  tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + col + (uint32_t)c0, v);
  tc_fence_before();
  __syncwarp();
  if (lane == 0) mbar_arrive(acc_empty);  // the values are in registers: the MMA may reuse the columns
#pragma unroll
  for (int h = 0; h < 32; h += 8) {
    const int j = (c0 + h) >> 3;  // the 16-byte chunk of the 128-byte row
    uint4* chunk = reinterpret_cast<uint4*>(out + r * 128 + ((j ^ (r & 7)) << 4));
    const uint4 m = mk[h >> 3];
    const uint32_t mw[4] = {m.x, m.y, m.z, m.w};
    uint32_t ow[4];
#pragma unroll
    for (int i = 0; i < 8; i += 2) {
      float z0 = v[h + i] + s_bias[c0 + h + i], z1 = v[h + i + 1] + s_bias[c0 + h + i + 1];
      if (a.relu) { z0 = fmaxf(z0, 0.f); z1 = fmaxf(z1, 0.f); }
      if (mrow) {  // keep where the forward activation (BF16) is positive
        if (!(__uint_as_float(mw[i >> 1] << 16) > 0.f)) z0 = 0.f;
        if (!(__uint_as_float(mw[i >> 1] & 0xffff0000u) > 0.f)) z1 = 0.f;
      }
      ow[i >> 1] = (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(z0)) |
                   ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(z1)) << 16);
    }
    *chunk = make_uint4(ow[0], ow[1], ow[2], ow[3]);
  }
}

// Tile i of this CTA is tile blockIdx.x + i gridDim.x (all roles walk the same list).
__global__ void __launch_bounds__(kConvThreads, 1)
    conv64_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
                     const ConvTcArgs a) {
  extern __shared__ __align__(128) unsigned char smem[];
  // everything from the next 1024-byte boundary (the 128-byte swizzle's period): the
  // weights, kStages tile buffers of kABytes and kOutBufs output staging tiles, each a
  // whole number of 1,024-byte atoms
  unsigned char* wsm = smem + ((1024u - (smem_u32(smem) & 1023u)) & 1023u);
  unsigned char* ring = wsm + kWBytes;
  unsigned char* obuf = ring + kStages * kABytes;
  __shared__ __align__(8) uint64_t full[kStages], empty[kStages], accf[kAcc], acce[kAcc], fin;
  __shared__ uint32_t tmem_base;
  __shared__ float s_bias[kC];
  __shared__ int s_fail;

  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_per_sample = a.len / kTileM;
  const int n_tiles = a.batch * tiles_per_sample;
  const int n_my = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  // resident weights (one bulk asynchronous copy, issued below with the first tiles) and
  // bias; barriers; TMEM
  __shared__ __align__(8) uint64_t wbar;
  if (tid < kC) s_bias[tid] = a.bias ? a.bias[tid] : 0.f;
  if (tid == 0) {
    for (int k = 0; k < kStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 1);
    }
    for (int k = 0; k < kAcc; ++k) {
      mbar_init(&accf[k], 1);
      mbar_init(&acce[k], kEpiWarps);  // one arrival per epilogue warp
    }
    mbar_init(&fin, 1);
    mbar_init(&wbar, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(&tmem_base, kAcc * kC);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;

  if (warp == 0 && lane == 0) {  // TMA producer
    mbar_arrive_expect_tx(&wbar, (uint32_t)kWBytes);
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(wsm)),
                 "l"(a.wpack), "r"((uint32_t)kWBytes), "r"(smem_u32(&wbar))
                 : "memory");
    int issued = 0;
    for (int i = 0; i < n_my && ok; ++i) {
      const int s = i % kStages;
      if (i >= kStages) ok = mbar_wait(&empty[s], (uint32_t)((i / kStages - 1) & 1), kWaitLimit);
      if (!ok) break;
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = t / tiles_per_sample, l0 = (t % tiles_per_sample) * kTileM;
      unsigned char* buf = ring + s * kABytes;
      mbar_arrive_expect_tx(&full[s], (uint32_t)kABytes);
      tma_load3(buf, &xmap, 0, l0 - kTaps / 2, b, &full[s]);
      issued = i + 1;
    }
    // every copy issued has landed before the CTA goes on (bounded)
    for (int i = issued > kStages ? issued - kStages : 0; i < issued; ++i)
      if (!mbar_wait(&full[i % kStages], (uint32_t)((i / kStages) & 1), kWaitLimit)) ok = false;
    if (!mbar_wait(&wbar, 0u, kWaitLimit)) ok = false;
  } else if (warp == 1 && lane == 0) {  // MMA issuer
    const uint32_t idesc = idesc_bf16_f32(kTileM, kC);
    // descriptors as a base plus a compile-time offset: every offset is a multiple of
    // 16 bytes and every address stays below 2^18, so (addr + off) >> 4 = (addr >> 4)
    // + (off >> 4) within the 14-bit start-address field
    const uint64_t bdesc0 = smem_desc_sw128(smem_u32(wsm));
    if (n_my > 0) ok = mbar_wait(&wbar, 0u, kWaitLimit);  // the weights have landed
    for (int i = 0; i < n_my && ok; ++i) {
      const int s = i % kStages, ac = i % kAcc;
      ok = mbar_wait(&full[s], (uint32_t)((i / kStages) & 1), kWaitLimit);
      if (ok && i >= kAcc) ok = mbar_wait(&acce[ac], (uint32_t)((i / kAcc - 1) & 1), kWaitLimit);
      if (!ok) break;
      tc_fence_after();
      const uint64_t adesc0 = smem_desc_sw128(smem_u32(ring + s * kABytes));
      const uint32_t dst = tmem + (uint32_t)(ac * kC);
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk) {
#pragma unroll
        for (int ks = 0; ks < kC / 16; ++ks) {  // tap kk: kk rows on; K step ks: 32 bytes along the row
          const uint64_t ad = adesc0 + (uint64_t)((kk * 128 + ks * 32) >> 4);
          const uint64_t bd = bdesc0 + (uint64_t)((kk * kC * 128 + ks * 32) >> 4);
          mma_bf16(dst, ad, bd, idesc, kk > 0 || ks > 0);
        }
      }
      mma_commit(&empty[s]);  // the buffer is free once these MMAs have read it
      mma_commit(&accf[ac]);  // the accumulator is ready
    }
    // every MMA issued has completed before TMEM is freed (bounded)
    mma_commit(&fin);
    if (!mbar_wait(&fin, 0u, kWaitLimit)) ok = false;
  } else if (warp >= 2) {  // epilogue: TMEM lane quarter warp % 4, channels c0 .. c0+31
    const int q = warp & 3, c0 = 32 * ((warp - 2) / 4);
    const bool issuer = warp == 2 && lane == 0;  // issues the tile's TMA store
    for (int i = 0; i < n_my; ++i) {
      const int ac = i % kAcc;
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      // staging tile i % 2: its store (tile i - 2) finished reading before the last barrier
      unsigned char* out = obuf + (i % kOutBufs) * kOutBytes;
      // the backward mask of this thread's row and channels, read before the wait so
      // that its latency overlaps the tile's MMAs
      uint4 mk[4] = {};
      if (a.mask) {
        const int l = (t % tiles_per_sample) * kTileM + 32 * q + lane;
        const uint4* mrow = reinterpret_cast<const uint4*>(
            a.mask + ((size_t)(t / tiles_per_sample) * a.len + l) * kC + c0);
#pragma unroll
        for (int h = 0; h < 4; ++h) mk[h] = __ldg(mrow + h);
      }
      bool mine = mbar_wait(&accf[ac], (uint32_t)((i / kAcc) & 1), kWaitLimit);
      mine = __all_sync(0xffffffffu, mine) != 0;
      if (mine) {
        tc_fence_after();
        conv_epilogue(a, s_bias, tmem, (uint32_t)(ac * kC), c0, q, &acce[ac], out, mk);
        fence_proxy_async_smem();  // the staged tile becomes visible to the TMA store
      }
      if (issuer) bulk_wait_read_all();  // tile i - 1's store has read the other staging tile
      ok = epi_barrier_and(mine);  // every epilogue warp takes the same branch
      if (!ok) break;
      if (issuer) tma_store3(&ymap, out, 0, (t % tiles_per_sample) * kTileM, t / tiles_per_sample);
    }
    if (issuer) bulk_wait_all();  // the stores are complete before the CTA ends
  }
  if (!ok) atomicExch(&s_fail, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (tid == 0 && s_fail) atomicOr(a.err, kErrMmaWait);
  if (warp == 1) tmem_dealloc(tmem, kAcc * kC);
}

// W[kk][co][ci] (FP32) -> BF16 planes for the tensor-core kernel. transpose=1
// packs the weights of the input-gradient convolution: W'[kk][ci][co] = W[8-kk][co][ci].
// Per tap kk, 64 rows n (the output channel) of 128 bytes (the 64 reduction channels),
// 16-byte chunk j of row n at chunk j ^ (n & 7): the MMA's 128-byte-swizzled layout.
__global__ void pack_w64_kernel(const float* w, uint4* out, int transpose) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (kk, row n, chunk j)
  if (i >= kTaps * kC * 8) return;
  const int kk = i / (kC * 8);
  const int n = (i / 8) % kC;
  const int j = i % 8;
  __align__(16) __nv_bfloat16 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) {
    const int k = 8 * j + e;  // reduction channel
    const float x = transpose ? w[((kTaps - 1 - kk) * kC + k) * kC + n] : w[(kk * kC + n) * kC + k];
    v[e] = __float2bfloat16_rn(x);
  }
  out[(kk * kC + n) * 8 + (j ^ (n & 7))] = *reinterpret_cast<const uint4*>(v);
}

// Shared memory of the conv kernel: resident weights, the row tiles and the output
// staging tiles (with up to 1 KB to align them).
int conv64_smem_bytes() { return kWBytes + kStages * kABytes + 1024 + kOutBufs * kOutBytes; }

// cuTensorMapEncodeTiled from the driver, found once through the runtime
static PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

int launch_conv64(const void* xv, const void* wv, const float* bias, const void* mv, void* yv,
                  int32_t* err, int batch, int len, int relu, void* stream) {
  const uint4* wpack = static_cast<const uint4*>(wv);
  const __nv_bfloat16* mask = static_cast<const __nv_bfloat16*>(mv);
  if (batch <= 0) return 0;
  // the input as a 3-D tensor (channel, position, sample), boxes of 64 channels x 136
  // rows x 1 sample (a whole tile, 128-byte swizzle), zeros outside the sample's [0, len)
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return (int)cudaErrorNotSupported;
  alignas(64) CUtensorMap map;
  const cuuint64_t dims[3] = {(cuuint64_t)kC, (cuuint64_t)len, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)kC * 2, (cuuint64_t)len * kC * 2};
  const cuuint32_t box[3] = {(cuuint32_t)kC, (cuuint32_t)kRows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(xv), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return (int)cudaErrorInvalidValue;
  // the output as the same 3-D tensor, boxes of a whole tile (64 channels x 128 rows),
  // 128-byte swizzle (one row of a tile is 128 bytes)
  alignas(64) CUtensorMap ymap;
  const cuuint32_t obox[3] = {(cuuint32_t)kC, (cuuint32_t)kTileM, 1};
  if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, yv, dims, strides, obox, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return (int)cudaErrorInvalidValue;
  const int smem = conv64_smem_bytes();
  cudaError_t e = cudaFuncSetAttribute(conv64_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return (int)e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = batch * (len / kTileM);
  const int grid = tiles < sms ? tiles : sms;
  ConvTcArgs a{wpack, bias, mask, err, batch, len, relu};
  conv64_tc_kernel<<<grid, kConvThreads, smem, (cudaStream_t)stream>>>(map, ymap, a);
  return (int)cudaGetLastError();
}

int launch_pack_w64(const float* w, void* out, int transpose, void* stream) {
  const int n = kTaps * kC * 8;
  pack_w64_kernel<<<(n + 127) / 128, 128, 0, (cudaStream_t)stream>>>(w, static_cast<uint4*>(out), transpose);
  return (int)cudaGetLastError();
}


// ------------------------------------------------------------------ other layers
// First layer QLP_CNN_IN_CH -> 64 channels and last layer 64 -> 1 channel (kernel 9, same
// padding) on the CUDA cores; their weight gradients and the bias gradients as
// two-stage reductions (per-CTA partial sums, then a sum over CTAs); BCE with
// logits; Adam with FP32 master weights.

// The small layers work on tiles of 128 positions of one sample (len is a multiple
// of 128): a CTA stages the tile's rows with the 4 halo rows on each side (zeros
// outside [0, len)) in shared memory and walks its tiles; 4 groups of 64 threads
// each take 32 consecutive positions, thread = channel, so that a position's 64
// channels are one coalesced 128-byte row and every row value a thread needs is
// read once into a sliding window of 9 rows held in registers (the loop over the
// group's 32 positions is unrolled, so the window's slots are fixed registers).
constexpr int kSmTile = 128;                      // positions per tile
constexpr int kSmRows = kSmTile + kTaps - 1;      // staged rows per tile
constexpr int kSmGroupPos = 32;                   // positions per thread group
constexpr int kSmThreads = 256;                   // 4 groups x 64 channels

// Tiles of the small-layer kernels and the CTAs that walk them.
__host__ __device__ __forceinline__ int small_tiles(int batch, int len) { return batch * (len / kSmTile); }

// x0 [B][L][CI] BF16 -> a1 [B][L][64] BF16 = relu(b1 + conv(x0, W1)), W1 [9][64][CI]:
// thread = output channel co, its 9 x CI weights in registers.
__global__ void __launch_bounds__(kSmThreads) conv_in_kernel(const __nv_bfloat16* x0, const float* w1,
                                                             const float* b1, __nv_bfloat16* a1, int batch,
                                                             int len) {
  constexpr int CI = QLP_CNN_IN_CH;
  __shared__ float s_x[kSmRows][CI];
  const int co = threadIdx.x & (kC - 1), g = threadIdx.x >> 6;
  float w[kTaps][CI];
#pragma unroll
  for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) w[kk][ci] = w1[(kk * kC + co) * CI + ci];
  const float bias = b1[co];
  const int tps = len / kSmTile, n_tiles = batch * tps;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int b = t / tps, l0 = (t - b * tps) * kSmTile;
    __syncthreads();  // the previous tile's rows are no longer read
    for (int i = threadIdx.x; i < kSmRows * CI; i += blockDim.x) {
      const int r = i / CI, ci = i - r * CI;
      const int l = l0 - kTaps / 2 + r;
      s_x[r][ci] = (l >= 0 && l < len) ? __bfloat162float(x0[((size_t)b * len + l) * CI + ci]) : 0.f;
    }
    __syncthreads();
    const int q0 = g * kSmGroupPos;
    float win[kTaps][CI];  // win[(q + kk) % 9] = staged row q0 + q + kk
#pragma unroll
    for (int r = 0; r < kTaps - 1; ++r)
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) win[r][ci] = s_x[q0 + r][ci];
    __nv_bfloat16* out = a1 + ((size_t)b * len + l0 + q0) * kC + co;
#pragma unroll
    for (int q = 0; q < kSmGroupPos; ++q) {
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) win[(q + kTaps - 1) % kTaps][ci] = s_x[q0 + q + kTaps - 1][ci];
      float z = bias;
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) z = fmaf(w[kk][ci], win[(q + kk) % kTaps][ci], z);
      out[(size_t)q * kC] = __float2bfloat16_rn(fmaxf(z, 0.f));
    }
  }
}

__device__ __forceinline__ void bf16x8_to_f32(uint4 u, float* f) {
  const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
  for (int e = 0; e < 8; ++e) f[e] = __bfloat162float(h[e]);
}

// a5 [B][L][64] BF16 -> logit [B][L] FP32 = b6 + conv(a5, W6), W6 [9][64]. Per staged
// row r and tap kk the CTA forms P[r][kk] = sum_ci W6[kk][ci] a5[r][ci] (thread = row,
// the row read once, the weights broadcast from shared memory), then logit[q] =
// b6 + sum_kk P[q + kk][kk]. Rows are 144 bytes apart in shared memory, so that a
// warp's 16-byte row reads fall in distinct bank groups.
constexpr int kOutRowB = 144;
__global__ void __launch_bounds__(160) conv_out_kernel(const __nv_bfloat16* a5, const float* w6,
                                                       const float* b6, float* logit, int batch, int len) {
  __shared__ __align__(16) unsigned char s_a[kSmRows * kOutRowB];
  __shared__ __align__(16) float s_w[kTaps * kC];
  __shared__ float s_p[kSmRows][kTaps + 1];
  for (int i = threadIdx.x; i < kTaps * kC; i += blockDim.x) s_w[i] = w6[i];
  const float bias = b6[0];
  const int tps = len / kSmTile, n_tiles = batch * tps;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int b = t / tps, l0 = (t - b * tps) * kSmTile;
    __syncthreads();
    for (int i = threadIdx.x; i < kSmRows * (kC / 8); i += blockDim.x) {
      const int r = i >> 3, c = i & 7;
      const int l = l0 - kTaps / 2 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (l >= 0 && l < len) v = reinterpret_cast<const uint4*>(a5 + ((size_t)b * len + l) * kC)[c];
      *reinterpret_cast<uint4*>(s_a + r * kOutRowB + c * 16) = v;
    }
    __syncthreads();
    if (threadIdx.x < kSmRows) {
      const int r = threadIdx.x;
      float acc[kTaps];
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk) acc[kk] = 0.f;
#pragma unroll
      for (int c = 0; c < kC / 8; ++c) {
        float f[8];
        bf16x8_to_f32(*reinterpret_cast<const uint4*>(s_a + r * kOutRowB + c * 16), f);
#pragma unroll
        for (int kk = 0; kk < kTaps; ++kk) {
          const float4 wa = *reinterpret_cast<const float4*>(s_w + kk * kC + 8 * c);
          const float4 wb = *reinterpret_cast<const float4*>(s_w + kk * kC + 8 * c + 4);
          acc[kk] = fmaf(wa.x, f[0], fmaf(wa.y, f[1], fmaf(wa.z, f[2], fmaf(wa.w, f[3], acc[kk]))));
          acc[kk] = fmaf(wb.x, f[4], fmaf(wb.y, f[5], fmaf(wb.z, f[6], fmaf(wb.w, f[7], acc[kk]))));
        }
      }
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk) s_p[r][kk] = acc[kk];
    }
    __syncthreads();
    if (threadIdx.x < kSmTile) {
      const int q = threadIdx.x;
      float z = bias;
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk) z += s_p[q + kk][kk];
      logit[(size_t)b * len + l0 + q] = z;
    }
  }
}

// Weighted BCE with logits, mean over B L: loss_i = pw y softplus(-z) + (1-y) softplus(z);
// dlogit_i = (pw y (sigmoid(z) - 1) + (1 - y) sigmoid(z)) / (B L).
__global__ void __launch_bounds__(256) bce_kernel(const float* logit, const float* label, float* dlogit,
                                                  float* loss, int n, float pos_weight) {
  __shared__ float red[8];
  float acc = 0.f;
  const float inv = 1.f / (float)n;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float z = logit[i], y = label[i];
    const float sp_pos = fmaxf(z, 0.f) + log1pf(expf(-fabsf(z)));  // softplus(z)
    const float sp_neg = sp_pos - z;                                // softplus(-z)
    acc += pos_weight * y * sp_neg + (1.f - y) * sp_pos;
    const float sg = 1.f / (1.f + expf(-z));
    dlogit[i] = (pos_weight * y * (sg - 1.f) + (1.f - y) * sg) * inv;
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    atomicAdd(loss, s * inv);
  }
}

// da5[b][l][ci] = (a5 > 0) * sum_kk W6[kk][ci] dlogit[b][l - kk + 4]: thread = (8-channel
// chunk, run of 8 consecutive positions of one sample), its 9 x 8 weights and the 16
// logit gradients around the run in registers; 8 threads cover a position's row.
constexpr int kBwdRun = 8;
__global__ void __launch_bounds__(256) conv_out_bwd_kernel(const float* dlogit, const float* w6,
                                                           const __nv_bfloat16* a5, __nv_bfloat16* da5,
                                                           int batch, int len) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (size_t)batch * len / kBwdRun * (kC / 8)) return;
  const int c = (int)(i & 7);
  const size_t p0 = (i >> 3) * kBwdRun;  // len is a multiple of kBwdRun: a run stays in one sample
  const int b = (int)(p0 / len), l0 = (int)(p0 - (size_t)b * len);
  float w[kTaps][8];
#pragma unroll
  for (int kk = 0; kk < kTaps; ++kk) {
    const float4 wa = *reinterpret_cast<const float4*>(w6 + kk * kC + 8 * c);
    const float4 wb = *reinterpret_cast<const float4*>(w6 + kk * kC + 8 * c + 4);
    w[kk][0] = wa.x; w[kk][1] = wa.y; w[kk][2] = wa.z; w[kk][3] = wa.w;
    w[kk][4] = wb.x; w[kk][5] = wb.y; w[kk][6] = wb.z; w[kk][7] = wb.w;
  }
  float d[kBwdRun + kTaps - 1];  // d[j] = dlogit[l0 - 4 + j], zero outside the sample
#pragma unroll
  for (int j = 0; j < kBwdRun + kTaps - 1; ++j) {
    const int ll = l0 - kTaps / 2 + j;
    d[j] = (ll >= 0 && ll < len) ? dlogit[(size_t)b * len + ll] : 0.f;
  }
#pragma unroll
  for (int j = 0; j < kBwdRun; ++j) {
    float s[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) s[e] = 0.f;
#pragma unroll
    for (int kk = 0; kk < kTaps; ++kk)  // dlogit[l - kk + 4] with l = l0 + j
#pragma unroll
      for (int e = 0; e < 8; ++e) s[e] = fmaf(w[kk][e], d[j + kTaps - 1 - kk], s[e]);
    const size_t p = p0 + j;
    float av[8];
    bf16x8_to_f32(reinterpret_cast<const uint4*>(a5 + p * kC)[c], av);
    __align__(16) __nv_bfloat16 o[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) o[e] = __float2bfloat16_rn(av[e] > 0.f ? s[e] : 0.f);
    reinterpret_cast<uint4*>(da5 + p * kC)[c] = *reinterpret_cast<const uint4*>(o);
  }
}

// Gradient outputs of a 64 -> 64 layer: dW [9][64][64] then db [64].
constexpr int kDwOut = kTaps * kC * kC + kC;

// Weight and bias gradients of a 64 -> 64 layer on the tensor cores:
//   dW[kk][co][ci] = sum_p dY[p][co] X[p + kk - 4][ci] = sum_q dY[q - kk + 4][co] X[q][ci],
// a GEMM over positions q (K) with M = output channel and N = input channel. A
// CTA walks 128-position tiles (K = 128 each) and accumulates all nine taps in
// TMEM across its tiles. Both operands are read "MN-major" from channels-last
// rows: 16 bytes = 8 consecutive channels of one position, one plane per 8
// channels with positions at a 16-byte stride, so a shift along positions is a
// shift of the descriptor's start address. Taps are paired in M = 128: rows
// 0..63 hold tap kk, rows 64..127 tap kk + 1, whose dY rows sit one position
// earlier; a second copy of the dY planes staged one row later makes that a
// single descriptor (planes 8..15 = planes 0..7 moved by one row). Pairs (0,1),
// (2,3), (4,5), (6,7), (8,-): 5 x 64 TMEM columns; the unused half of the last
// pair reads staged rows and is discarded.
// Warp roles: warp 0 loads each tile with TMA (24 boxes of 8 channels x 136 rows:
// dY from the tile's row - 4 and - 5, X from its row; zeros outside the sample)
// into a ring of 4 buffers; one thread of warp 1 issues the tile's 40 MMAs and
// commits them to the buffer's empty barrier; warps 2-3 add the tile's own dY
// rows into the bias gradient (thread = output channel) and arrive on the same
// barrier. After the last tile all four warps read the accumulators (lane
// quarter = warp) into the CTA's partial sums.
constexpr int kWgTile = 128;                     // positions per tile (K)
constexpr int kWgRows = kWgTile + kTaps - 1;     // 136 staged rows per plane (dY and X)
constexpr int kWgPlane = kWgRows * 16;           // 2,176 B
constexpr int kWgABytes = 2 * kPlanes * kWgPlane;  // 16 dY planes: 34,816 B
constexpr int kWgBBytes = kPlanes * kWgPlane;    // 8 X planes: 17,408 B
constexpr int kWgStage = kWgABytes + kWgBBytes;  // 52,224 B per stage
constexpr int kWgStages = 4;
constexpr int kWgPairs = 5;
constexpr int kWgThreads = 128;
constexpr int kWgSmem = kWgStages * kWgStage;    // 208,896 B: one CTA per SM (512 TMEM columns)

__global__ void __launch_bounds__(kWgThreads, 1)
    wgrad64_tc_kernel(const __grid_constant__ CUtensorMap dymap, const __grid_constant__ CUtensorMap xmap,
                      float* partial, int32_t* err, int batch, int len) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[kWgStages], empty[kWgStages], fin;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  const int tiles_per_sample = len / kWgTile;
  const int n_tiles = batch * tiles_per_sample;
  const int n_my = (int)blockIdx.x < n_tiles ? (n_tiles - 1 - (int)blockIdx.x) / (int)gridDim.x + 1 : 0;

  if (tid == 0) {
    for (int k = 0; k < kWgStages; ++k) {
      mbar_init(&full[k], 1);
      mbar_init(&empty[k], 3);  // the MMAs' commit and the two bias warps
    }
    mbar_init(&fin, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) tmem_alloc(&tmem_base, 512);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = tmem_base;
  bool ok = true;
  float db = 0.f;

  if (warp == 0 && lane == 0) {  // TMA producer
    int issued = 0;
    for (int i = 0; i < n_my && ok; ++i) {
      const int s = i % kWgStages;
      if (i >= kWgStages) ok = mbar_wait(&empty[s], (uint32_t)((i / kWgStages - 1) & 1), kWaitLimit);
      if (!ok) break;
      const int t = (int)blockIdx.x + i * (int)gridDim.x;
      const int b = t / tiles_per_sample, q0 = (t % tiles_per_sample) * kWgTile;
      unsigned char* buf = smem + s * kWgStage;
      mbar_arrive_expect_tx(&full[s], (uint32_t)kWgStage);
#pragma unroll
      for (int j = 0; j < kPlanes; ++j) {
        tma_load3(buf + j * kWgPlane, &dymap, 8 * j, q0 - kTaps / 2, b, &full[s]);
        tma_load3(buf + (kPlanes + j) * kWgPlane, &dymap, 8 * j, q0 - kTaps / 2 - 1, b, &full[s]);
        tma_load3(buf + kWgABytes + j * kWgPlane, &xmap, 8 * j, q0, b, &full[s]);
      }
      issued = i + 1;
    }
    for (int i = issued > kWgStages ? issued - kWgStages : 0; i < issued; ++i)  // every copy has landed
      if (!mbar_wait(&full[i % kWgStages], (uint32_t)((i / kWgStages) & 1), kWaitLimit)) ok = false;
  } else if (warp == 1 && lane == 0) {  // MMA issuer: M = 128, N = 64, A and B MN-major
    const uint32_t idesc = idesc_bf16_f32(128, kC) | (1u << 15) | (1u << 16);
    for (int i = 0; i < n_my && ok; ++i) {
      const int s = i % kWgStages;
      ok = mbar_wait(&full[s], (uint32_t)((i / kWgStages) & 1), kWaitLimit);
      if (!ok) break;
      tc_fence_after();
      const uint32_t abase = smem_u32(smem + s * kWgStage), bbase = abase + kWgABytes;
#pragma unroll 1
      for (int g = 0; g < kWgPairs; ++g) {
        const int kk = 2 * g;
#pragma unroll
        for (int ks = 0; ks < kWgTile / 16; ++ks) {
          const uint64_t ad = smem_desc(abase + (uint32_t)((kTaps - 1 - kk) * 16 + ks * 256), 128, kWgPlane);
          const uint64_t bd = smem_desc(bbase + (uint32_t)(ks * 256), 128, kWgPlane);
          mma_bf16(tmem + (uint32_t)(g * kC), ad, bd, idesc, i > 0 || ks > 0);
        }
      }
      mma_commit(&empty[s]);  // the buffer is free once these MMAs have read it
    }
    mma_commit(&fin);  // every MMA issued has completed before TMEM is read or freed (bounded)
    if (!mbar_wait(&fin, 0u, kWaitLimit)) ok = false;
  } else if (warp >= 2) {  // bias gradient: the tile's own dY rows (staged rows 4 .. 131 of plane co / 8)
    const int co = tid - 64;
    for (int i = 0; i < n_my && ok; ++i) {
      const int s = i % kWgStages;
      ok = mbar_wait(&full[s], (uint32_t)((i / kWgStages) & 1), kWaitLimit);
      ok = __all_sync(0xffffffffu, ok) != 0;
      if (!ok) break;
      const unsigned char* col = smem + s * kWgStage + (co >> 3) * kWgPlane + (co & 7) * 2;
#pragma unroll 8
      for (int r = kTaps / 2; r < kTaps / 2 + kWgTile; ++r)
        db += __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(col + r * 16));
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
    }
  }
  if (!ok) atomicExch(&s_fail, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  float* out = partial + (size_t)blockIdx.x * kDwOut;
  if (!s_fail && n_my > 0) {
    // TMEM lane m = 32 warp + lane: tap 2g + (m >= 64), output channel m % 64; column = input channel
    const int m = 32 * warp + lane;
    const int co = m & (kC - 1);
#pragma unroll 1
    for (int g = 0; g < kWgPairs; ++g) {
      const int kk = 2 * g + (m >= kC ? 1 : 0);
#pragma unroll
      for (int c0 = 0; c0 < kC; c0 += 16) {
        float v[16];
        tmem_ld16(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(g * kC + c0), v);
        if (kk < kTaps) {
          float4* dst = reinterpret_cast<float4*>(out + (kk * kC + co) * kC + c0);
          dst[0] = make_float4(v[0], v[1], v[2], v[3]);
          dst[1] = make_float4(v[4], v[5], v[6], v[7]);
          dst[2] = make_float4(v[8], v[9], v[10], v[11]);
          dst[3] = make_float4(v[12], v[13], v[14], v[15]);
        }
      }
    }
    if (warp >= 2) out[kTaps * kC * kC + (tid - 64)] = db;
  } else if (!s_fail) {  // no tiles: zero partial sums
    for (int i = tid; i < kDwOut; i += kWgThreads) out[i] = 0.f;
  } else if (tid == 0) {
    atomicOr(err, kErrMmaWait);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

// Partial gradients of a small layer: n_co x n_ci channels (first layer 64 x QLP_CNN_IN_CH with
// dY BF16, last layer 1 x 64 with dY FP32). One thread per (kk, co, ci) output
// plus n_co bias outputs; each CTA covers a range of positions.
template <typename TY>
__global__ void __launch_bounds__(256) dw_small_kernel(const TY* dy, const __nv_bfloat16* x, float* partial,
                                                       int batch, int len, int n_co, int n_ci, int per_cta) {
  const int n_w = kTaps * n_co * n_ci;
  const int n_out = n_w + n_co;
  const int total = batch * len;
  const int p_begin = blockIdx.x * per_cta;
  const int p_end = min(total, p_begin + per_cta);
  for (int o = threadIdx.x; o < n_out; o += blockDim.x) {
    float acc = 0.f;
    if (o < n_w) {
      const int kk = o / (n_co * n_ci), co = (o / n_ci) % n_co, ci = o % n_ci;
      for (int p = p_begin; p < p_end; ++p) {
        const int b = p / len, l = p - b * len;
        const int ll = l + kk - kTaps / 2;
        if (ll < 0 || ll >= len) continue;
        acc += (float)dy[(size_t)p * n_co + co] * __bfloat162float(x[((size_t)b * len + ll) * n_ci + ci]);
      }
    } else {
      const int co = o - n_w;
      for (int p = p_begin; p < p_end; ++p) acc += (float)dy[(size_t)p * n_co + co];
    }
    partial[(size_t)blockIdx.x * n_out + o] = acc;
  }
}

// Per-CTA partial gradients of the first layer (64 x QLP_CNN_IN_CH channels, dY BF16):
// dW1[kk][co][ci] = sum_q dY[q][co] X[q + kk - 4][ci], db1[co] = sum_q dY[q][co]. Thread
// = output channel co of one group; the 9 x CI input values around q in a sliding
// window of registers, 9 x CI accumulators. The groups' sums are added in shared
// memory in group order, then written as the CTA's partial.
__global__ void __launch_bounds__(kSmThreads) dw_in_kernel(const __nv_bfloat16* dy, const __nv_bfloat16* x,
                                                           float* partial, int batch, int len) {
  constexpr int CI = QLP_CNN_IN_CH, NW = kTaps * CI;
  __shared__ float s_x[kSmRows][CI];
  __shared__ float s_red[kSmThreads / kC - 1][kC][NW + 1];  // the sums of groups 1..3
  const int co = threadIdx.x & (kC - 1), g = threadIdx.x >> 6;
  float acc[kTaps][CI];
#pragma unroll
  for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
    for (int ci = 0; ci < CI; ++ci) acc[kk][ci] = 0.f;
  float acc_b = 0.f;
  const int tps = len / kSmTile, n_tiles = batch * tps;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int b = t / tps, l0 = (t - b * tps) * kSmTile;
    __syncthreads();
    for (int i = threadIdx.x; i < kSmRows * CI; i += blockDim.x) {
      const int r = i / CI, ci = i - r * CI;
      const int l = l0 - kTaps / 2 + r;
      s_x[r][ci] = (l >= 0 && l < len) ? __bfloat162float(x[((size_t)b * len + l) * CI + ci]) : 0.f;
    }
    __syncthreads();
    const int q0 = g * kSmGroupPos;
    float win[kTaps][CI];
#pragma unroll
    for (int r = 0; r < kTaps - 1; ++r)
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) win[r][ci] = s_x[q0 + r][ci];
    const __nv_bfloat16* drow = dy + ((size_t)b * len + l0 + q0) * kC + co;
#pragma unroll
    for (int q = 0; q < kSmGroupPos; ++q) {
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) win[(q + kTaps - 1) % kTaps][ci] = s_x[q0 + q + kTaps - 1][ci];
      const float a = __bfloat162float(drow[(size_t)q * kC]);
      acc_b += a;
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
        for (int ci = 0; ci < CI; ++ci) acc[kk][ci] = fmaf(a, win[(q + kk) % kTaps][ci], acc[kk][ci]);
    }
  }
  if (g > 0) {
#pragma unroll
    for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) s_red[g - 1][co][kk * CI + ci] = acc[kk][ci];
    s_red[g - 1][co][NW] = acc_b;
  }
  __syncthreads();
  if (g == 0) {  // group 0 adds the others' sums to its own, in group order
    float* out = partial + (size_t)blockIdx.x * (kTaps * kC * CI + kC);
#pragma unroll
    for (int kk = 0; kk < kTaps; ++kk)
#pragma unroll
      for (int ci = 0; ci < CI; ++ci) {
        float v = acc[kk][ci];
        for (int gg = 0; gg < kSmThreads / kC - 1; ++gg) v += s_red[gg][co][kk * CI + ci];
        out[(kk * kC + co) * CI + ci] = v;
      }
    float v = acc_b;
    for (int gg = 0; gg < kSmThreads / kC - 1; ++gg) v += s_red[gg][co][NW];
    out[kTaps * kC * CI + co] = v;
  }
}

// Per-CTA partial gradients of the last layer (64 -> 1, dY FP32):
// dW6[kk][ci] = sum_q dY[q] A5[q + kk - 4][ci], db6 = sum_q dY[q]. Thread = input channel ci
// of one group; the 9 values of its channel around q in a sliding window, 9 accumulators.
__global__ void __launch_bounds__(kSmThreads) dw_out_kernel(const float* dy, const __nv_bfloat16* x,
                                                            float* partial, int batch, int len) {
  __shared__ float s_dy[kSmTile];
  __shared__ __align__(16) __nv_bfloat16 s_a[kSmRows][kC];
  __shared__ float s_red[kSmThreads / kC][kC][kTaps + 1];
  const int ci = threadIdx.x & (kC - 1), g = threadIdx.x >> 6;
  float acc[kTaps];
#pragma unroll
  for (int kk = 0; kk < kTaps; ++kk) acc[kk] = 0.f;
  float acc_b = 0.f;
  const int tps = len / kSmTile, n_tiles = batch * tps;
  for (int t = blockIdx.x; t < n_tiles; t += gridDim.x) {
    const int b = t / tps, l0 = (t - b * tps) * kSmTile;
    __syncthreads();
    for (int i = threadIdx.x; i < kSmTile; i += blockDim.x) s_dy[i] = dy[(size_t)b * len + l0 + i];
    for (int i = threadIdx.x; i < kSmRows * (kC / 8); i += blockDim.x) {
      const int r = i >> 3, c = i & 7;
      const int l = l0 - kTaps / 2 + r;
      uint4 v = make_uint4(0u, 0u, 0u, 0u);
      if (l >= 0 && l < len) v = reinterpret_cast<const uint4*>(x + ((size_t)b * len + l) * kC)[c];
      *reinterpret_cast<uint4*>(&s_a[r][8 * c]) = v;
    }
    __syncthreads();
    const int q0 = g * kSmGroupPos;
    float win[kTaps];
#pragma unroll
    for (int r = 0; r < kTaps - 1; ++r) win[r] = __bfloat162float(s_a[q0 + r][ci]);
#pragma unroll
    for (int q = 0; q < kSmGroupPos; ++q) {
      win[(q + kTaps - 1) % kTaps] = __bfloat162float(s_a[q0 + q + kTaps - 1][ci]);
      const float d = s_dy[q0 + q];
      if (ci == 0) acc_b += d;
#pragma unroll
      for (int kk = 0; kk < kTaps; ++kk) acc[kk] = fmaf(d, win[(q + kk) % kTaps], acc[kk]);
    }
  }
#pragma unroll
  for (int kk = 0; kk < kTaps; ++kk) s_red[g][ci][kk] = acc[kk];
  s_red[g][ci][kTaps] = acc_b;
  __syncthreads();
  float* out = partial + (size_t)blockIdx.x * (kTaps * kC + 1);
  for (int i = threadIdx.x; i < kTaps * kC + 1; i += blockDim.x) {
    float v = 0.f;
    if (i < kTaps * kC) {
      const int kk = i / kC, c = i - kk * kC;
      for (int gg = 0; gg < kSmThreads / kC; ++gg) v += s_red[gg][c][kk];
    } else {
      for (int gg = 0; gg < kSmThreads / kC; ++gg) v += s_red[gg][0][kTaps];
    }
    out[i] = v;
  }
}

// out[o] = sum over the CTA partials g of partial[g][o]: a CTA takes 32 outputs, its 8
// warps the partials g = w, w + 8, ... (in that order), then warp 0 adds the 8 sums in
// warp order (a fixed order: deterministic).
constexpr int kRedSlices = 8;
__global__ void __launch_bounds__(32 * kRedSlices) reduce_partials_kernel(const float* partial, int n_parts,
                                                                         int n_out, float* out) {
  __shared__ float red[kRedSlices][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int o = blockIdx.x * 32 + lane;
  float s = 0.f;
  if (o < n_out)
    for (int g = w; g < n_parts; g += kRedSlices) s += partial[(size_t)g * n_out + o];
  red[w][lane] = s;
  __syncthreads();
  if (w == 0 && o < n_out) {
    float t = 0.f;
    for (int k = 0; k < kRedSlices; ++k) t += red[k][lane];
    out[o] = t;
  }
}
static void launch_reduce_partials(const float* partial, int n_parts, int n_out, float* out, cudaStream_t s) {
  reduce_partials_kernel<<<(n_out + 31) / 32, 32 * kRedSlices, 0, s>>>(partial, n_parts, n_out, out);
}

// Adam with the decay rates and their complements given separately (each the
// FP32 rounding of its exact decimal value: 1 - 0.999f is 1.3e-5 away from 0.001)
// and the bias corrections c1 = 1 - b1^t, c2 = 1 - b2^t computed in FP64 by the host.
__global__ void adam_kernel(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2,
                            float omb1, float omb2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + omb1 * gi;
  const float vi = b2 * v[i] + omb2 * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// ------------------------------------------------------------------ launchers

// CTAs of a small-layer kernel: a few per SM, each walking its share of the tiles
static int small_grid(int batch, int len, int per_sm) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = small_tiles(batch, len);
  return tiles < per_sm * sms ? tiles : per_sm * sms;
}

int launch_conv_in(const void* x0, const float* w1, const float* b1, void* a1, int batch, int len, void* s) {
  if (batch <= 0 || len % kSmTile != 0) return batch <= 0 ? 0 : (int)cudaErrorInvalidValue;
  conv_in_kernel<<<small_grid(batch, len, 2), kSmThreads, 0, (cudaStream_t)s>>>(
      static_cast<const __nv_bfloat16*>(x0), w1, b1, static_cast<__nv_bfloat16*>(a1), batch, len);
  return (int)cudaGetLastError();
}

int launch_conv_out(const void* a5, const float* w6, const float* b6, float* logit, int batch, int len, void* s) {
  if (batch <= 0 || len % kSmTile != 0) return batch <= 0 ? 0 : (int)cudaErrorInvalidValue;
  conv_out_kernel<<<small_grid(batch, len, 8), 160, 0, (cudaStream_t)s>>>(static_cast<const __nv_bfloat16*>(a5),
                                                                          w6, b6, logit, batch, len);
  return (int)cudaGetLastError();
}

int launch_bce(const float* logit, const float* label, float* dlogit, float* loss, int n, float pw, void* s) {
  const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
  bce_kernel<<<blocks, 256, 0, (cudaStream_t)s>>>(logit, label, dlogit, loss, n, pw);
  return (int)cudaGetLastError();
}

int launch_conv_out_bwd(const float* dlogit, const float* w6, const void* a5, void* da5, int batch, int len,
                        void* s) {
  if (len % kBwdRun != 0) return (int)cudaErrorInvalidValue;
  const size_t n = (size_t)batch * len / kBwdRun * (kC / 8);
  if (n == 0) return 0;
  conv_out_bwd_kernel<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)s>>>(
      dlogit, w6, static_cast<const __nv_bfloat16*>(a5), static_cast<__nv_bfloat16*>(da5), batch, len);
  return (int)cudaGetLastError();
}

int dw_small_parts(int batch, int len) {
  const int total = batch * len;
  return (total + 1023) / 1024 < 512 ? (total + 1023) / 1024 : 512;
}


int wgrad64_parts(int batch, int len) {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int tiles = batch * (len / kWgTile);
  return tiles < sms ? tiles : sms;
}

// dW and db of a 64 -> 64 layer on the tensor cores (len a multiple of 128):
// per-CTA partial sums, then their sum into out[kDwOut]
int launch_wgrad64(const void* dy, const void* x, float* partial, float* out, int32_t* err, int batch, int len,
                   void* s) {
  if (batch <= 0) return 0;
  const int parts = wgrad64_parts(batch, len);
  // dY and X as 3-D tensors (channel, position, sample), boxes of 8 channels x 136 rows
  PFN_cuTensorMapEncodeTiled_v12000 enc = encode_tiled();
  if (!enc) return (int)cudaErrorNotSupported;
  alignas(64) CUtensorMap dymap, xmap;
  const cuuint64_t dims[3] = {(cuuint64_t)kC, (cuuint64_t)len, (cuuint64_t)batch};
  const cuuint64_t strides[2] = {(cuuint64_t)kC * 2, (cuuint64_t)len * kC * 2};
  const cuuint32_t box[3] = {8, (cuuint32_t)kWgRows, 1};
  const cuuint32_t estr[3] = {1, 1, 1};
  if (enc(&dymap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(dy), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS ||
      enc(&xmap, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void*>(x), dims, strides, box, estr,
          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return (int)cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(wgrad64_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kWgSmem);
  if (e != cudaSuccess) return (int)e;
  wgrad64_tc_kernel<<<parts, kWgThreads, kWgSmem, (cudaStream_t)s>>>(dymap, xmap, partial, err, batch, len);
  launch_reduce_partials(partial, parts, kDwOut, out, (cudaStream_t)s);
  return (int)cudaGetLastError();
}

// dW and db of the first (dy BF16 [B][L][64], x BF16 [B][L][QLP_CNN_IN_CH]) or last (dy FP32
// [B][L], x BF16 [B][L][64]) layer into out[9 co ci + co]
int launch_dw_small(const void* dy, int dy_is_f32, const void* x, float* partial, float* out, int batch,
                    int len, int n_co, int n_ci, void* s) {
  const int total = batch * len;
  int parts = dw_small_parts(batch, len);
  int per = (total + parts - 1) / parts;
  const int n_out = kTaps * n_co * n_ci + n_co;
  const bool tiled = len % kSmTile == 0;
  if (tiled) {  // no more CTAs than the partial buffer holds
    const int g = small_grid(batch, len, 2);
    parts = g < parts ? g : parts;
  }
  if (tiled && !dy_is_f32 && n_co == kC && n_ci == QLP_CNN_IN_CH) {  // the first layer
    dw_in_kernel<<<parts, kSmThreads, 0, (cudaStream_t)s>>>(static_cast<const __nv_bfloat16*>(dy),
                                                             static_cast<const __nv_bfloat16*>(x), partial, batch,
                                                             len);
  } else if (tiled && dy_is_f32 && n_co == 1 && n_ci == kC) {  // the last layer
    dw_out_kernel<<<parts, kSmThreads, 0, (cudaStream_t)s>>>(static_cast<const float*>(dy),
                                                              static_cast<const __nv_bfloat16*>(x), partial, batch,
                                                              len);
  } else if (dy_is_f32)
    dw_small_kernel<float><<<parts, 256, 0, (cudaStream_t)s>>>(static_cast<const float*>(dy),
                                                                static_cast<const __nv_bfloat16*>(x), partial,
                                                                batch, len, n_co, n_ci, per);
  else
    dw_small_kernel<__nv_bfloat16><<<parts, 256, 0, (cudaStream_t)s>>>(
        static_cast<const __nv_bfloat16*>(dy), static_cast<const __nv_bfloat16*>(x), partial, batch, len, n_co,
        n_ci, per);
  launch_reduce_partials(partial, parts, n_out, out, (cudaStream_t)s);
  return (int)cudaGetLastError();
}

int launch_adam(float* p, const float* g, float* m, float* v, int n, float lr, float b1, float b2, float omb1,
                float omb2, float eps, float c1, float c2, void* s) {
  adam_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)s>>>(p, g, m, v, n, lr, b1, b2, omb1, omb2, eps, c1, c2);
  return (int)cudaGetLastError();
}

}  // namespace qlp
