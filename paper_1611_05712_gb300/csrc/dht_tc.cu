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
// Precision (two kinds): 3-term TF32 products (every float x split as hi = x rounded to
// TF32 and lo = x - hi, D accumulates Xhi*Ahi + Xhi*Alo + Xlo*Ahi) or 6-term BF16 products
// (x split into three BF16 pieces, the six products of order <= 2); FP32 accumulation in
// tensor memory; the matrices' pieces are precomputed from their FP64 values at setup.
//
// Kernel: persistent and warp-specialised (k_dht_tc_ws): one CTA per SM walks the
// (M tile, N tile, batch) tiles; producer warps stage the panel and issue the matrix
// copies into a ring of shared-memory stages, one thread issues the MMAs into one of two
// TMEM accumulators, and epilogue warps drain the other accumulator (tcgen05.ld, warp w
// owns TMEM lanes 32*(w%4)..+31, stores of 32 consecutive c per warp), so a tile's
// epilogue runs under the next tile's main loop.  Every mbarrier wait is bounded and sets
// the device error word on timeout.
#include <cuda.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "pic_internal.cuh"
#include "tc_common.cuh"

namespace pic {
namespace {

constexpr int kTcM = 128;          // rows of D (columns c of Xf) per CTA
constexpr int kTcMaxN = 256;       // largest N tile, TF32 form
constexpr int kTcMaxNBf16 = 128;   // largest N tile, BF16 form (three planes per operand)

struct TcParams {
  int Nr;        // K extent and rows of A
  int Nc;        // columns of Xf (2 Nz)
  int NT;        // N tile (multiple of 16, <= 256)
  int n_tiles;   // N tiles per batch
  int tmem_cols; // power of two >= max(32, NT)
  int m_tiles;   // 128-column tiles per batch
};

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

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// The two product kinds.  Planes are the pieces an operand is split into; product p
// multiplies A plane a_plane[p] by B plane b_plane[p].
//   TF32x3: x = hi + lo (hi = x rounded to TF32), products hi.hi, hi.lo, lo.hi;
//   BF16x6: x = b0 + b1 + b2 (each the BF16 rounding of what is left), products of order
//           <= 2: b0.b0, b0.b1, b1.b0, b0.b2, b1.b1, b2.b0.
// A 128-byte swizzle row holds 128 / kElemBytes elements; one MMA consumes 32 bytes of K.
template <int KIND> struct TcKind;
template <> struct TcKind<0> {
  static constexpr int kPlanes = 2, kElemBytes = 4, kProducts = 3;
  static constexpr uint32_t kIdesc = (1u << 4) | (2u << 7) | (2u << 10);   // D f32, A/B tf32
  __device__ static int a_plane(int p) { return p == 2 ? 1 : 0; }
  __device__ static int b_plane(int p) { return p == 1 ? 1 : 0; }
  __device__ static void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    mma_tf32(d, a, b, idesc, acc);
  }
};
template <> struct TcKind<1> {
  static constexpr int kPlanes = 3, kElemBytes = 2, kProducts = 6;
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

// ---- persistent, warp-specialised form ------------------------------------------------
// One CTA per SM walks the tiles (m fastest, then n, then batch) with a stride of the grid.
//   warps 0-7 (producers): each thread owns half of one row c of the 128-row M tile; per K
//     chunk it splits its prefetched panel values and writes them swizzled into the stage,
//     then the warp arrives on full[stage]; thread 0 first arms full[stage] with the matrix
//     tiles' transaction bytes and issues their TMA copies.  The next chunk's loads (of this
//     or the next tile) are issued before the wait for a free stage.
//   warp 12 (MMA): one thread waits full[stage], issues the products into the tile's
//     accumulator (two TMEM accumulators of N_T columns, alternating by tile), commits to
//     empty[stage], and after a tile's last chunk commits to tmem_full[acc].
//   warps 8-11 (epilogue): wait tmem_full[acc], read their 32 TMEM lanes (rows c) with
//     tcgen05.ld and store Y, then arrive on tmem_empty[acc]; the MMA thread waits on it
//     before it reuses that accumulator two tiles later.
// So a tile's epilogue runs under the next tile's main loop.  Every wait is bounded; a
// timeout sets the device error word and a shared abort flag that every loop checks, and
// before tensor memory is released the CTA waits (bounded) for its copies and MMAs.
constexpr int kWsThreads = 416;   // 8 producer warps, 4 epilogue warps, 1 MMA warp
constexpr int kWsMaxStages = 4;

struct WsTile {
  int b, n0, c0;
};

__device__ __forceinline__ WsTile ws_tile(int t, const TcParams& P) {
  const int m = t % P.m_tiles;
  const int rest = t / P.m_tiles;
  return WsTile{rest / P.n_tiles, (rest % P.n_tiles) * P.NT, m * kTcM};
}

template <int KIND>
__global__ void __launch_bounds__(kWsThreads, 1) k_dht_tc_ws(DhtBatch bt, TcParams P,
                                                              const __grid_constant__ TcMaps maps, int32_t* err,
                                                              int n_stages, int n_tiles_total) {
  using K = TcKind<KIND>;
  constexpr int NP = K::kPlanes;
  constexpr int EPC = 16 / K::kElemBytes;    // K elements per 16-byte chunk of a swizzle row
  constexpr int KPR = 8 * EPC;              // K elements per 128-byte row (= kChunkK)
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const uint32_t a_bytes = kTcM * 128;
  const uint32_t b_bytes = (uint32_t)P.NT * 128;
  const uint32_t stage_bytes = NP * (a_bytes + b_bytes);
  uint64_t* full = reinterpret_cast<uint64_t*>(base + n_stages * stage_bytes);
  uint64_t* empty = full + kWsMaxStages;
  uint64_t* tfull = empty + kWsMaxStages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nK = (P.Nr + KPR - 1) / KPR;
  const uint32_t tmem_cols = (uint32_t)P.tmem_cols;

  if (warp == 12) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < n_stages; ++i) {
      mbar_init(&full[i], 9);    // TMA issuer's arrive.expect_tx + one arrival per producer warp
      mbar_init(&empty[i], 1);   // MMA commit
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);   // MMA commit after a tile's last chunk
      mbar_init(&tempty[i], 4);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  const uint32_t idesc = K::kIdesc | ((uint32_t)(P.NT >> 3) << 17) | ((uint32_t)(kTcM >> 4) << 24);

  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(err, kErrTimeout);
  };

  if (warp < 8) {
    // ---------------------------------------------------------------- producers
    constexpr int HALF = KPR / 2;   // K elements (4 swizzle chunks) per thread and chunk
    const int row = tid & (kTcM - 1);
    const int half = tid >> 7;      // which 4 of the row's 8 16-byte chunks
    float pv[HALF];
    auto load = [&](int t, int kc) {
      const WsTile w = ws_tile(t, P);
      const float* __restrict__ X = static_cast<const float*>(bt.X[w.b]);
      const int c = w.c0 + row;
#pragma unroll
      for (int e = 0; e < HALF; ++e) {
        const int j = kc * KPR + half * HALF + e;
        pv[e] = (c < P.Nc && j < P.Nr) ? X[(size_t)j * P.Nc + c] : 0.f;
      }
    };
    uint32_t g = 0;
    int last_armed = -1;   // stage armed by thread 0 whose bytes may still be in flight
    bool have = blockIdx.x < n_tiles_total && nK > 0;
    if (have) load(blockIdx.x, 0);
    for (int t = blockIdx.x; t < n_tiles_total && !*abort_flag; t += gridDim.x) {
      const WsTile w = ws_tile(t, P);
      for (int kc = 0; kc < nK; ++kc, ++g) {
        const int st = (int)(g % (uint32_t)n_stages);
        const uint32_t use = g / (uint32_t)n_stages;
        if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1)) { fail(); break; }
        if (*abort_flag) break;
        unsigned char* sA = base + st * stage_bytes;
        unsigned char* sB = sA + NP * a_bytes;
        if (tid == 0) {
          mbar_arrive_expect_tx(&full[st], NP * b_bytes);
#pragma unroll
          for (int pl = 0; pl < NP; ++pl) tma_load_2d(sB + pl * b_bytes, &maps.m[pl][w.b], kc * KPR, w.n0, &full[st]);
          last_armed = st;
        }
#pragma unroll
        for (int cq = 0; cq < 4; ++cq) {
          const int ch = half * 4 + cq;
          const uint32_t off = sw128_off(row, ch);
          if (KIND == 0) {
            float hv[4], lv[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              hv[e] = tf32_hi(pv[cq * 4 + e]);
              lv[e] = pv[cq * 4 + e] - hv[e];
            }
            *reinterpret_cast<float4*>(sA + off) = make_float4(hv[0], hv[1], hv[2], hv[3]);
            *reinterpret_cast<float4*>(sA + a_bytes + off) = make_float4(lv[0], lv[1], lv[2], lv[3]);
          } else {
            uint32_t w0[4], w1[4], w2[4];
#pragma unroll
            for (int e = 0; e < 8; e += 2) {
              uint32_t a0, a1, a2, b0, b1, b2;
              split_bf16x3(pv[cq * 8 + e], a0, a1, a2);
              split_bf16x3(pv[cq * 8 + e + 1], b0, b1, b2);
              w0[e / 2] = a0 | (b0 << 16);
              w1[e / 2] = a1 | (b1 << 16);
              w2[e / 2] = a2 | (b2 << 16);
            }
            *reinterpret_cast<uint4*>(sA + off) = make_uint4(w0[0], w0[1], w0[2], w0[3]);
            *reinterpret_cast<uint4*>(sA + a_bytes + off) = make_uint4(w1[0], w1[1], w1[2], w1[3]);
            *reinterpret_cast<uint4*>(sA + 2 * a_bytes + off) = make_uint4(w2[0], w2[1], w2[2], w2[3]);
          }
        }
        // the next chunk's panel values: of this tile, or the first of the next tile
        if (kc + 1 < nK) load(t, kc + 1);
        else if (t + (int)gridDim.x < n_tiles_total) load(t + gridDim.x, 0);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(&full[st]);
      }
    }
    // before shared memory is released: the last armed stage's copies must have landed
    if (tid == 0 && last_armed >= 0 && *abort_flag) {
      const uint32_t gl = g == 0 ? 0 : g - 1;
      mbar_wait(&full[last_armed], (gl / (uint32_t)n_stages) & 1);
    }
  } else if (warp == 12) {
    // ---------------------------------------------------------------- MMA issuer
    if (lane == 0) {
      uint32_t g = 0, i = 0;
      uint64_t* last_bar = nullptr;   // barrier and phase of the last commit issued
      uint32_t last_parity = 0;
      for (int t = blockIdx.x; t < n_tiles_total && !*abort_flag; t += gridDim.x, ++i) {
        const uint32_t acc = i & 1, acc_use = i >> 1;
        if (acc_use > 0 && !mbar_wait(&tempty[acc], (acc_use - 1) & 1)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + acc * (uint32_t)P.NT;
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int st = (int)(g % (uint32_t)n_stages);
          if (!mbar_wait(&full[st], (g / (uint32_t)n_stages) & 1)) { fail(); ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + st * stage_bytes), sb = sa + NP * a_bytes;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks) {
            const uint32_t koff = ks * 32;
#pragma unroll
            for (int pr = 0; pr < K::kProducts; ++pr) {
              const uint32_t accf = (kc > 0 || ks > 0 || pr > 0) ? 1u : 0u;
              K::mma(d, make_desc(sa + K::a_plane(pr) * a_bytes + koff), make_desc(sb + K::b_plane(pr) * b_bytes + koff),
                     idesc, accf);
            }
          }
          mma_commit(&empty[st]);
          last_bar = &empty[st];
          last_parity = (g / (uint32_t)n_stages) & 1;
        }
        if (!ok) break;
        mma_commit(&tfull[acc]);
        last_bar = &tfull[acc];
        last_parity = (i >> 1) & 1;
      }
      // on abort: let the MMAs already issued finish before tensor memory is released
      if (*abort_flag && last_bar) mbar_wait(last_bar, last_parity);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue (warps 8-11)
    const int q = warp - 8;   // TMEM lanes 32q..32q+31 = rows c (warp % 4 == q)
    uint32_t i = 0;
    for (int t = blockIdx.x; t < n_tiles_total && !*abort_flag; t += gridDim.x, ++i) {
      const uint32_t acc = i & 1;
      if (!mbar_wait(&tfull[acc], (i >> 1) & 1)) { fail(); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const WsTile w = ws_tile(t, P);
      float* __restrict__ Y = static_cast<float*>(bt.Y[w.b]);
      const int c = w.c0 + q * 32 + lane;
      for (int j0 = 0; j0 < P.NT; j0 += 8) {
        uint32_t r[8];
        const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)P.NT + (uint32_t)j0;
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
            : "r"(taddr)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c < P.Nc) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int n = w.n0 + j0 + e;
            if (n < P.Nr) Y[(size_t)n * P.Nc + c] = __uint_as_float(r[e]);
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 12)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
}

// Health check of the bounded waits: an mbarrier that nothing arrives on, waited on with a
// cap of max_polls polls; the timeout raises the error bit and the kernel returns.
__global__ void k_wait_selftest(int32_t* err, uint32_t max_polls) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    const uint32_t a = smem_u32(&bar);
    bool done = false;
    for (uint32_t it = 0; it < max_polls && !done; ++it) {
      uint32_t d;
      asm volatile(
          "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
          : "=r"(d)
          : "r"(a), "r"(0u)
          : "memory");
      done = d != 0;
    }
    if (!done) atomicOr(err, kErrTimeout);
  }
}

}  // namespace

constexpr size_t kWsSmemMax = 227 * 1024;   // dynamic shared memory of the persistent kernel
int sm_count_of[64] = {};

// SMs of the current device (recorded by dht_tc_configure_device).
int dht_tc_sm_count() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64 || sm_count_of[dev] <= 0) return 152;
  return sm_count_of[dev];
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
  PIC_CUDA(cudaFuncSetAttribute(k_dht_tc_ws<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemMax));
  PIC_CUDA(cudaFuncSetAttribute(k_dht_tc_ws<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWsSmemMax));
  int sms = 0;
  PIC_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (dev >= 0 && dev < 64) sm_count_of[dev] = sms;
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

void* tensor_map_encoder() { return reinterpret_cast<void*>(encode_fn()); }

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
  // persistent, warp-specialised launch: one CTA per SM, as many stages as shared memory
  // holds (2..4), two TMEM accumulators of N_T columns
  const int planes = bf ? 3 : 2;
  const size_t stage_bytes = (size_t)planes * (kTcM * 128 + (size_t)P.NT * 128);
  const int n_stages = (int)std::min<size_t>(kWsMaxStages, (kWsSmemMax - 1024 - 128) / stage_bytes);
  if (n_stages < 2) {
    set_error("DHT tile N=%d does not fit two stages in shared memory", P.NT);
    return PIC_ERR_ARG;
  }
  int tc2 = 32;
  while (tc2 < 2 * P.NT) tc2 <<= 1;
  P.tmem_cols = tc2;
  const int n_tiles_total = P.m_tiles * P.n_tiles * b.n;
  const int grid = std::min(n_tiles_total, dht_tc_sm_count());
  const size_t smem = 1024 + (size_t)n_stages * stage_bytes + 128;
  if (bf)
    k_dht_tc_ws<1><<<grid, kWsThreads, smem, s->stream>>>(b, P, maps, s->at<int32_t>(s->lay.err), n_stages,
                                                          n_tiles_total);
  else
    k_dht_tc_ws<0><<<grid, kWsThreads, smem, s->stream>>>(b, P, maps, s->at<int32_t>(s->lay.err), n_stages,
                                                          n_tiles_total);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_wait_selftest(Sim* s, uint32_t max_polls) {
  k_wait_selftest<<<1, 32, 0, s->stream>>>(s->at<int32_t>(s->lay.err), max_polls);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
