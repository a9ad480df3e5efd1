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
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kTcThreads = 256;
constexpr int kTcM = 128;          // rows of D (columns c of Xf) per CTA
constexpr int kTcK = 32;           // floats of K per stage (128 bytes = one swizzle row)
constexpr int kTcMaxN = 256;
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

// Instruction descriptor, kind::tf32: D f32, A/B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t make_idesc(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
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

// Tensor maps of the batch's split matrices (hi, lo), passed by value as a grid constant.
struct TcMaps {
  Sim::TensorMapBytes hi[24];
  Sim::TensorMapBytes lo[24];
};

__global__ void __launch_bounds__(kTcThreads, 1) k_dht_tc(DhtBatch bt, TcParams P, const __grid_constant__ TcMaps maps,
                                                           int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up: [stage][A_hi | A_lo | B_hi | B_lo], then barriers
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t a_bytes = kTcM * 128;            // 16 KB
  const uint32_t b_bytes = (uint32_t)P.NT * 128;  // up to 32 KB
  const uint32_t stage_bytes = 2 * a_bytes + 2 * b_bytes;
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
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.hi[b])) : "memory");
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&maps.lo[b])) : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = make_idesc(kTcM, P.NT);
  const int nK = (P.Nr + kTcK - 1) / kTcK;
  bool ok = true;
  int issued = -1, committed = -1;   // last chunk whose matrix copies / MMAs were issued (block-uniform)

  // data-panel values of the next chunk, loaded ahead of the wait for a free stage:
  // item it = tid + q*256 covers row c0 + (it % 128), 16-byte chunk it / 128 (4 values of j)
  float pv[4][4];
  auto load_chunk = [&](int kc) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = tid + q * kTcThreads;
      const int c = c0 + (it & (kTcM - 1)), ch = it >> 7;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int j = kc * kTcK + ch * 4 + e;
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
    unsigned char* sA = base + st * stage_bytes;
    unsigned char* sAlo = sA + a_bytes;
    unsigned char* sB = sAlo + a_bytes;
    unsigned char* sBlo = sB + b_bytes;
    const int k0 = kc * kTcK;
    if (tid == 0) {   // matrix tiles (rows n0.., columns k0..k0+31; zero fill beyond Nr)
      mbar_arrive_expect_tx(&bars[2 + st], 2 * b_bytes);
      tma_load_2d(sB, &maps.hi[b], k0, n0, &bars[2 + st]);
      tma_load_2d(sBlo, &maps.lo[b], k0, n0, &bars[2 + st]);
    }
    issued = kc;
    // A operand (transposed X): split the prefetched values and store them swizzled
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int it = tid + q * kTcThreads;
      const int row = it & (kTcM - 1), ch = it >> 7;
      float hv[4], lv[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        hv[e] = tf32_hi(pv[q][e]);
        lv[e] = pv[q][e] - hv[e];
      }
      const uint32_t off = sw128_off(row, ch);
      *reinterpret_cast<float4*>(sA + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
      *reinterpret_cast<float4*>(sAlo + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
    }
    if (kc + 1 < nK) load_chunk(kc + 1);   // in flight while this chunk is multiplied
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const bool landed = (tid == 0) ? mbar_wait(&bars[2 + st], (uint32_t)((kc >> 1) & 1)) : true;
    if (!__syncthreads_and(landed)) { ok = false; break; }
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a_hi = smem_u32(sA), a_lo = smem_u32(sAlo), b_hi = smem_u32(sB), b_lo = smem_u32(sBlo);
#pragma unroll
      for (int ks = 0; ks < kTcK / 8; ++ks) {
        const uint32_t koff = ks * 32;   // 8 tf32 = 32 bytes along K inside the swizzle row
        const uint32_t acc0 = (kc > 0 || ks > 0) ? 1u : 0u;
        mma_tf32(tmem, make_desc(a_hi + koff), make_desc(b_hi + koff), idesc, acc0);
        mma_tf32(tmem, make_desc(a_hi + koff), make_desc(b_lo + koff), idesc, 1u);
        mma_tf32(tmem, make_desc(a_lo + koff), make_desc(b_hi + koff), idesc, 1u);
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

size_t dht_tc_smem_bytes(int NT) { return 1024 + 2 * (2 * kTcM * 128 + 2 * (size_t)NT * 128) + 64; }

// Raised once per device to the largest tile (N_T = 256); per-launch changes of this
// per-function attribute would race between host threads.
pic_status dht_tc_configure_device() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PIC_OK;
  PIC_CUDA(cudaFuncSetAttribute(k_dht_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)dht_tc_smem_bytes(kTcMaxN)));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

namespace {

// N tiling shared by the tensor maps and the launches: n_tiles tiles of NT rows of A
// (the tuned tile if set, else Nr split into the fewest tiles of <= 256 rows).
void tc_tiles(const Sim* s, int* n_tiles, int* NT) {
  const int Nr = s->cfg.Nr;
  if (s->tune_nt > 0) {
    *NT = std::min(s->tune_nt, (Nr + 15) / 16 * 16);
    *n_tiles = (Nr + *NT - 1) / *NT;
    return;
  }
  *n_tiles = (Nr + kTcMaxN - 1) / kTcMaxN;
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

// Tensor maps of the split matrices: 2-D float32 views (Nr columns j, Nr rows n, row
// pitch split_pitch(Nr)), box 32 j x NT rows, 128-byte swizzle; coordinates past Nr read 0.
pic_status dht_tc_make_maps(Sim* s) {
  std::memset(s->tmaps, 0, sizeof(s->tmaps));
  if (s->cfg.precision == PIC_FP64) return PIC_OK;
  EncodeTiledFn encode = encode_fn();
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PIC_ERR_CUDA;
  }
  const int Nr = s->cfg.Nr, pitch = split_pitch(Nr);
  int n_tiles = 0, NT = 0;
  tc_tiles(s, &n_tiles, &NT);
  const size_t mat_floats = (size_t)Nr * pitch;
  for (int dir = 0; dir < 2; ++dir) {
    for (int mi = 0; mi < s->cfg.Nm * 3; ++mi) {
      for (int part = 0; part < 2; ++part) {
        const size_t off = dir == 0 ? (part == 0 ? s->lay.mfwd_hi : s->lay.mfwd_lo)
                                    : (part == 0 ? s->lay.binv_hi : s->lay.binv_lo);
        float* g = s->at<float>(off) + (size_t)mi * mat_floats;
        const cuuint64_t dims[2] = {(cuuint64_t)Nr, (cuuint64_t)Nr};
        const cuuint64_t strides[1] = {(cuuint64_t)pitch * sizeof(float)};
        const cuuint32_t box[2] = {(cuuint32_t)kTcK, (cuuint32_t)NT};
        const cuuint32_t estr[2] = {1, 1};
        CUtensorMap* map = reinterpret_cast<CUtensorMap*>(s->tmaps[dir * kMaxModes * 3 + mi][part].b);
        const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, g, dims, strides, box, estr,
                                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
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
    maps.hi[i] = s->tmaps[b.mat[i]][0];
    maps.lo[i] = s->tmaps[b.mat[i]][1];
  }
  const size_t smem = dht_tc_smem_bytes(P.NT);
  dim3 grid(P.m_tiles, P.n_tiles, b.n);
  k_dht_tc<<<grid, kTcThreads, smem, s->stream>>>(b, P, maps, s->at<int32_t>(s->lay.err));
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
