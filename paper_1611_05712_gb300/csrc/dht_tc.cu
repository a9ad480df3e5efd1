// DHT of the mixed-precision form on the 5th-generation tensor cores (tcgen05, sm_103a).
//
// The discrete Hankel transform along r (section "Finite order pseudo-spectral solvers":
// Hankel transform along r) is, per (component, mode) pair, Y = A X with A the Nr x Nr
// real matrix and X the Nr x Nz complex panel, i.e. Xf (Nr x 2Nz floats, re/im
// interleaved).  Here it is computed transposed,
//     D[c][n] = sum_j Xf[j][c] A[n][j]      (D = Yf^T, M = columns c, N = rows n, K = j),
// so both tensor-core operands are K-major: the A-operand tile (128 columns c x 32 j) is
// transposed while it is staged into shared memory by the CTA's threads, and the B operand
// (rows of A, K-major as stored, row pitch a multiple of 16 bytes) is copied by the tensor
// memory accelerator (2-D tiled copies, completion counted in mbarrier transaction bytes;
// coordinates past Nr read zero).  Both use the 128-byte swizzled canonical layout.
//
// Precision: 3-term TF32 products.  Every float operand x is split as hi = x rounded to
// TF32 and lo = x - hi (exact in float); D accumulates Xhi*Ahi + Xhi*Alo + Xlo*Ahi in FP32
// in tensor memory (the A split is precomputed from the FP64 matrix at setup).
//
// One CTA owns a 128-column x N_T tile of D (N_T <= 256 TMEM columns) for one batch; K is
// consumed in chunks of 32 through two shared-memory stages: all 256 threads stage chunk
// k+1 while the tensor core runs chunk k, and the data-panel loads of chunk k+2 are issued
// before the wait for chunk k+1's stage.  One thread issues the MMAs and commits them to
// an mbarrier per stage; every wait on an mbarrier is bounded and sets the device error
// word on timeout.  The epilogue reads TMEM with tcgen05.ld (warp w owns TMEM lanes
// 32*(w%4)..+31) and writes Yf[n][c] so that the 32 lanes of a warp store 32 consecutive c.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;          // rows of D (columns c of Xf) per CTA
constexpr int kTcMaxN = 256;       // largest N tile, TF32 form
constexpr int kTcMaxNBf16 = 128;   // largest N tile, BF16 form (three planes per operand)
constexpr uint32_t kTcWaitCap = 1u << 26;   // mbarrier polls before giving up

struct TcParams {
  int Nr;        // K extent and rows of A
  int Nc;        // columns of Xf (2 Nz)
  int NT;        // N tile (multiple of 16, <= 256)
  int n_tiles;   // N tiles per batch
  int tmem_cols; // power of two >= max(32, NT)
  int m_tiles;   // 128-column tiles per batch
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of 16-byte chunk `ch` (0..7) of row `row` in a K-major SW128 tile.
__device__ __forceinline__ uint32_t sw128_off(int row, int ch) {
  return (uint32_t)((row >> 3) * 1024 + (row & 7) * 128 + ((ch ^ (row & 7)) << 4));
}

// SM100 shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 B apart.
__device__ __forceinline__ uint64_t make_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);          // start address
  d |= (uint64_t)1u << 16;                          // leading byte offset (unused for SW128 K-major)
  d |= (uint64_t)(1024u >> 4) << 32;                // stride byte offset: 8 rows x 128 B
  d |= (uint64_t)1u << 46;                          // descriptor version (SM100)
  d |= (uint64_t)2u << 61;                          // layout: SWIZZLE_128B
  return d;
}

__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t b = __float_as_uint(x);
  b = (b + 0x0fffu + ((b >> 13) & 1u)) & 0xffffe000u;   // round to nearest even at bit 13
  return __uint_as_float(b);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Bounded wait for completion `parity` of an mbarrier; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  for (uint32_t it = 0; it < kTcWaitCap; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                        uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The two product kinds.  Planes are the pieces an operand is split into; product p
// multiplies A plane a_plane[p] by B plane b_plane[p].
//   TF32x3: x = hi + lo (hi = x rounded to TF32), products hi.hi, hi.lo, lo.hi;
//   BF16x6: x = b0 + b1 + b2 (each the BF16 rounding of what is left), products of order
//           <= 2: b0.b0, b0.b1, b1.b0, b0.b2, b1.b1, b2.b0.
// A 128-byte swizzle row holds kChunkK elements; one MMA consumes 32 bytes of K.
template <int KIND> struct TcKind;
template <> struct TcKind<0> {
  static constexpr int kPlanes = 2, kElemBytes = 4, kChunkK = 32, kProducts = 3;
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10);   // D f32, A/B tf32
  __device__ static int a_plane(int p) { return p == 2 ? 1 : 0; }
  __device__ static int b_plane(int p) { return p == 1 ? 1 : 0; }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_tf32(d, a, b, idesc, acc);
  }
};
template <> struct TcKind<1> {
  static constexpr int kPlanes = 3, kElemBytes = 2, kChunkK = 64, kProducts = 6;
  static constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10);   // D f32, A/B bf16
  __device__ static int a_plane(int p) { return (p == 2 || p == 4) ? 1 : (p == 5 ? 2 : 0); }
  __device__ static int b_plane(int p) { return (p == 1 || p == 4) ? 1 : (p == 3 ? 2 : 0); }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_f16(d, a, b, idesc, acc);
  }
};

// x = b0 + b1 + b2 with each piece the BF16 rounding of what is left (differences exact in
// float); returns the three 16-bit patterns.
__device__ __forceinline__ void split_bf16x3(float x, uint32_t& b0, uint32_t& b1, uint32_t& b2) {
  const __nv_bfloat16 h0 = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h0);
  const __nv_bfloat16 h1 = __float2bfloat16_rn(r1);
  const float r2 = r1 - __bfloat162float(h1);
  b0 = __bfloat16_as_ushort(h0);
  b1 = __bfloat16_as_ushort(h1);
  b2 = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// One arrival on `bar` that also expects `bytes` of asynchronous-copy transactions.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// 2-D tiled tensor copy global -> shared (box at inner coordinate x, row y), completing
// its bytes on `bar`.  x is a multiple of 32 floats, so the start is 128-byte aligned.
__device__ __forceinline__ void tma_load_2d(void* dst, const void* tmap, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Tensor maps of the batch's split matrices (one per plane), passed by value as a grid
// constant.
struct TcMaps {
  Sim::TensorMapBytes m[3][24];
};

template <int KIND>
__global__ void __launch_bounds__(kTcThreads, 1) k_dht_tc(DhtBatch bt, TcParams P, const __grid_constant__ TcMaps maps,
                                                           int32_t* err) {
  using K = TcKind<KIND>;
  constexpr int NP = K::kPlanes;
  constexpr int EPC = 16 / K::kElemBytes;   // K elements per 16-byte chunk of a swizzle row
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up: [stage][A planes | B planes], then barriers
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t a_bytes = kTcM * 128;            // 16 KB per plane
  const uint32_t b_bytes = (uint32_t)P.NT * 128;  // up to 32 KB per plane
  const uint32_t stage_bytes = NP * (a_bytes + b_bytes);
  // bars[0..1]: per-stage "MMAs that read this stage are done"; bars[2..3]: per-stage
  // "matrix tiles have landed" (transaction counted)
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + 2 * stage_bytes);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 4);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int b = blockIdx.z;
  const int n_tile = blockIdx.y;
  const int m_tile = blockIdx.x;
  const int c0 = m_tile * kTcM, n0 = n_tile * P.NT;
  const float* __restrict__ X = static_cast<const float*>(bt.X[b]);
  float* __restrict__ Y = static_cast<float*>(bt.Y[b]);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"((uint32_t)P.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    mbar_init(&bars[3], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
    for (int pl = 0; pl < NP; ++pl)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.m[pl][b])) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = K::kIdesc | ((uint32_t)(P.NT >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);
  const int nK = (P.Nr + K::kChunkK - 1) / K::kChunkK;
  bool ok = true;
  int issued = -1, committed = -1;   // last chunk whose matrix copies / MMAs were issued (block-uniform)

  // data-panel values of the next chunk, loaded ahead of the wait for a free stage:
  // item it = tid + q*256 covers row c0 + (it % 128), 16-byte chunk it / 128 (EPC values of j)
  float pv[4][EPC];
  auto load_chunk = [&](int kc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = tid + q * kTcThreads;
      const int c = c0 + (it & (kTcM - 1)), ch = it >> 7;
#pragma unroll
      for (int e = 0; e < EPC; ++e) {
        const int j = kc * K::kChunkK + ch * EPC + e;
        pv[q][e] = (c < P.Nc && j < P.Nr) ? X[(size_t)j * P.Nc + c] : 0.f;
      }
    }
  };
  if (nK > 0) load_chunk(0);

  for (int kc = 0; kc < nK && ok; ++kc) {
    const int st = kc & 1;
    if (kc >= 2) {   // the MMAs that last read this stage (chunk kc-2) must be done
      const bool w = mbar_wait(&bars[st], (uint32_t)(((kc - 2) >> 1) & 1));
      if (!__syncthreads_and(w)) { ok = false; break; }   // one decision for the whole block
    }
    unsigned char* sA = base + st * stage_bytes;      // NP planes of a_bytes
    unsigned char* sB = sA + NP * a_bytes;            // NP planes of b_bytes
    const int k0 = kc * K::kChunkK;
    if (tid == 0) {   // matrix tiles (rows n0.., columns k0..; zero fill beyond Nr)
      mbar_arrive_expect_tx(&bars[2 + st], NP * b_bytes);
#pragma unroll
      for (int pl = 0; pl < NP; ++pl) tma_load_2d(sB + pl * b_bytes, &maps.m[pl][b], k0, n0, &bars[2 + st]);
    }
    issued = kc;
    // A operand (transposed X): split the prefetched values and store them swizzled
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = tid + q * kTcThreads;
      const int row = it & (kTcM - 1), ch = it >> 7;
      const uint32_t off = sw128_off(row, ch);
      if (KIND == 0) {
        float hv[4], lv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          hv[e] = tf32_hi(pv[q][e]);
          lv[e] = pv[q][e] - hv[e];
        }
        *reinterpret_cast<float4*>(sA + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
        *reinterpret_cast<float4*>(sA + a_bytes + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
      } else {
        uint32_t w0[4], w1[4], w2[4];
#pragma unroll
        for (int e = 0; e < EPC; e += 2) {
          uint32_t a0, a1, a2, b0, b1, b2;
          split_bf16x3(pv[q][e], a0, a1, a2);
          split_bf16x3(pv[q][e + 1], b0, b1, b2);
          w0[e / 2] = a0 | (b0 << 16);
          w1[e / 2] = a1 | (b1 << 16);
          w2[e / 2] = a2 | (b2 << 16);
        }
        *reinterpret_cast<uint4*>(sA + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
        *reinterpret_cast<uint4*>(sA + a_bytes + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
        *reinterpret_cast<uint4*>(sA + 2 * a_bytes + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
      }
    }
    if (kc + 1 < nK) load_chunk(kc + 1);   // in flight while this chunk is multiplied
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const bool landed = (tid == 0) ? mbar_wait(&bars[2 + st], (uint32_t)((kc >> 1) & 1)) : true;
    if (!__syncthreads_and(landed)) { ok = false; break; }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = smem_u32(sA), sb = smem_u32(sB);
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint32_t koff = ks * 32;   // 32 bytes of K per MMA inside the swizzle row
#pragma unroll
        for (int pr = 0; pr < K::kProducts; ++pr) {
          const uint32_t acc = (kc > 0 || ks > 0 || pr > 0) ? 1u : 0u;
          K::mma(tmem, make_desc(sa + K::a_plane(pr) * a_bytes + koff), make_desc(sb + K::b_plane(pr) * b_bytes + koff),
                 idesc, acc);
        }
      }
      mma_commit(&bars[st]);
    }
    committed = kc;
  }
  // wait for the last chunk's commit (it covers every MMA issued before it)
  if (ok && nK > 0) ok = mbar_wait(&bars[(nK - 1) & 1], (uint32_t)(((nK - 1) >> 1) & 1));
  ok = __syncthreads_and(ok);
  if (!ok) {
    if (tid == 0) {
      atomicOr(err, kErrTimeout);
      // wait (bounded) for the copies and MMAs still in flight before the shared and
      // tensor memory are released
      if (issued > committed) mbar_wait(&bars[2 + (issued & 1)], (uint32_t)((issued >> 1) & 1));
      if (committed >= 0) mbar_wait(&bars[committed & 1], (uint32_t)((committed >> 1) & 1));
    }
    __syncthreads();
  }
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");

  if (ok) {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (rows c) and half (w/4) of the N columns
    const int quarter = warp & 3, half = warp >> 2;
    const int c = c0 + quarter * 32 + lane;
    const int ncol_half = P.NT / 2;
    for (int j0 = half * ncol_half; j0 < (half + 1) * ncol_half; j0 += 8) {
      uint32_t r[8];
      const uint32_t taddr = tmem + ((uint32_t)(quarter * 32) << 16) + (uint32_t)j0;
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
          : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
          : "r"(taddr)
          : "memory");
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (c < P.Nc) {
#pragma unroll
        for (int e = 0; e < 8; ++e) {
          const int n = n0 + j0 + e;
          if (n < P.Nr) Y[(size_t)n * P.Nc + c] = __uint_as_float(r[e]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)P.tmem_cols)
                 : "memory");
}

}  // namespace

// Dynamic shared memory of one launch: two stages of planes x (A tile + B tile), barriers.
size_t dht_tc_smem_bytes(int planes, int NT) {
  return 1024 + 2 * (size_t)planes * (kTcM * 128 + (size_t)NT * 128) + 64;
}

// Raised once per device to the largest tile of each kind (TF32: N_T = 256, BF16: 128);
// per-launch changes of this per-function attribute would race between host threads.
pic_status dht_tc_configure_device() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PIC_OK;
  PIC_CUDA(cudaFuncSetAttribute(k_dht_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dht_tc_smem_bytes(2, kTcMaxN)));
  PIC_CUDA(cudaFuncSetAttribute(k_dht_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dht_tc_smem_bytes(3, kTcMaxNBf16)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

namespace {

bool is_bf16(const Sim* s) { return s->cfg.precision == PIC_MIXED_BF16X6; }

// N tiling shared by the tensor maps and the launches: n_tiles tiles of NT rows of A
// (the tuned tile if set, else Nr split into the fewest tiles of <= 256 rows, or <= 128
// in the BF16 form, whose three planes per operand fill shared memory at 128).
void tc_tiles(const Sim* s, int* n_tiles, int* NT) {
  const int Nr = s->cfg.Nr;
  const int cap = is_bf16(s) ? kTcMaxNBf16 : kTcMaxN;
  if (s->tune_nt > 0) {
    *NT = std::min(std::min(s->tune_nt, cap), (Nr + 15) / 16 * 16);
    *n_tiles = (Nr + *NT - 1) / *NT;
    return;
  }
  *n_tiles = (Nr + cap - 1) / cap;
  const int per = (Nr + *n_tiles - 1) / *n_tiles;
  *NT = (per + 15) / 16 * 16;
}

using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

}  // namespace

// Tensor maps of the split matrices: 2-D views of each plane (Nr columns j, Nr rows n,
// rows padded to 16 bytes), box of one 128-byte swizzle row of j (32 float or 64 BF16
// elements) x NT rows, 128-byte swizzle; coordinates past Nr read 0.
pic_status dht_tc_make_maps(Sim* s) {
  std::memset(s->tmaps, 0, sizeof(s->tmaps));
  if (s->cfg.precision == PIC_FP64) return PIC_OK;
  EncodeTiledFn encode = encode_fn();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PIC_ERR_CUDA;
  }
  const bool bf = is_bf16(s);
  const int Nr = s->cfg.Nr;
  const int pitch = bf ? split_pitch_b16(Nr) : split_pitch(Nr);
  const size_t esz = bf ? 2 : 4;
  const int planes = bf ? 3 : 2;
  int n_tiles = 0, NT = 0;
  tc_tiles(s, &n_tiles, &NT);
  const size_t mat_bytes = (size_t)Nr * pitch * esz;
  const size_t plane_bytes = (size_t)s->cfg.Nm * 3 * mat_bytes;   // BF16: planes follow each other
  for (int dir = 0; dir < 2; ++dir) {
    for (int mi = 0; mi < s->cfg.Nm * 3; ++mi) {
      for (int part = 0; part < planes; ++part) {
        char* g;
        if (bf) {
          g = s->at<char>(dir == 0 ? s->lay.mfwd_hi : s->lay.binv_hi) + part * plane_bytes + mi * mat_bytes;
        } else {
          const size_t off = dir == 0 ? (part == 0 ? s->lay.mfwd_hi : s->lay.mfwd_lo)
                                      : (part == 0 ? s->lay.binv_hi : s->lay.binv_lo);
          g = s->at<char>(off) + mi * mat_bytes;
        }
        const cuuint64_t dims[2] = {(cuuint64_t)Nr, (cuuint64_t)Nr};
        const cuuint64_t strides[1] = {(cuuint64_t)pitch * esz};
        const cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)NT};
        const cuuint32_t estr[2] = {1, 1};
        CUtensorMap* map = reinterpret_cast<CUtensorMap*>(s->tmaps[dir * kMaxModes * 3 + mi][part].b);
        const CUresult r = encode(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                                  g, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
          set_error("cuTensorMapEncodeTiled failed (%d) for split matrix %d", (int)r, dir * kMaxModes * 3 + mi);
          return PIC_ERR_CUDA;
        }
      }
    }
  }
  return PIC_OK;
}

pic_status launch_dht_tc(Sim* s, const DhtBatch& b) {
  const int Nr = s->cfg.Nr, Nc = 2 * s->cfg.Nz;
  const bool bf = is_bf16(s);
  TcParams P;
  P.Nr = Nr;
  P.Nc = Nc;
  tc_tiles(s, &P.n_tiles, &P.NT);
  int tc = 32;
  while (tc < P.NT) tc <<= 1;
  P.tmem_cols = tc;
  P.m_tiles = (Nc + kTcM - 1) / kTcM;
  TcMaps maps;
  for (int i = 0; i < b.n; ++i) {
    if (b.mat[i] < 0 || b.mat[i] >= 2 * kMaxModes * 3) {
      set_error("DHT batch entry %d has no split matrix", i);
      return PIC_ERR_ARG;
    }
    for (int pl = 0; pl < 3; ++pl) maps.m[pl][i] = s->tmaps[b.mat[i]][pl];
  }
  dim3 grid(P.m_tiles, P.n_tiles, b.n);
  if (bf)
    k_dht_tc<1><<<grid, kTcThreads, dht_tc_smem_bytes(3, P.NT), s->stream>>>(b, P, maps, s->at<int32_t>(s->lay.err));
  else
    k_dht_tc<0><<<grid, kTcThreads, dht_tc_smem_bytes(2, P.NT), s->stream>>>(b, P, maps, s->at<int32_t>(s->lay.err));
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
