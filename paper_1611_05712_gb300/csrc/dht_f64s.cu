// DHT of the FP64 form on the 5th-generation tensor cores, with FP64 results.
//
// The discrete Hankel transform along r (section "Finite order pseudo-spectral solvers":
// Hankel transform along r) is, per (component, mode) pair, Y = A X with A the Nr x Nr
// FP64 matrix and X the Nr x 2Nz FP64 panel.  GB300 runs FP64 arithmetic at 1/64 of its
// FP32 rate and far below its tensor rate, so this path computes the product exactly in
// pieces on the BF16 tensor cores and combines them in FP64 (the splitting idea of Ozaki
// et al., "Error-free transformations of matrix multiplication by using fast routines of
// matrix multiplication and its applications", Numer. Algorithms 59, 2012, here with
// fixed-width integer slices):
//   * every row n of A and every column c of X is scaled by a power of two, 2^E_n and
//     2^E_c, so that its entries lie in (-1, 1); the scaled value v is cut into S = 7
//     slices of W = 7 bits, v = sum_i s_i 2^(-W (i+1)) + r with integers |s_i| <= 127 (the
//     magnitude truncated to 49 bits, |r| < 2^-49), each exactly a BF16 number;
//   * a slice product sum over K <= 256 terms is an integer below 256 * 2^14 = 2^22, and
//     up to four such sums add up to at most 2^24: the tensor cores' FP32 accumulators
//     hold them exactly.  Group g collects the products a_i x_j with i + j = g (weight
//     2^(-W (g+2))): groups 0..3 (at most 4 products each) are exact, groups 4..6 add an
//     FP32 rounding of relative size 2^-24 at weight <= 2^-42; products with i + j >= S
//     are left out (weight <= 2^-63);
//   * the epilogue combines the 7 group accumulators in 64-bit integer arithmetic,
//     converts once to FP64 and scales by 2^(E_c + E_n).
// The result agrees with the FP64 product to about 2^-49 of max|A_n| max|X_c| K.  Used
// for Nr <= 256 (the exactness bound above); larger Nr keep the FP64 SIMT GEMM.
//
// Pieces: k_f64s_matrix slices the matrices at set-up (7 BF16 planes each, K-major);
// per DHT k_f64s_colmax finds the column maxima and k_f64s_panel slices the panels
// into K-major planes; k_dht_f64s is a persistent warp-specialised tcgen05 kernel: one
// thread issues the tensor-memory-access copies of both operands (7 planes each, 64-byte
// swizzle, 32 K elements per stage) into a ring of stages, three threads (one per warp,
// each owning whole groups) issue the 28 slice products per 16 K elements into 7 TMEM
// accumulators of a 128 x 64 tile, and 16 epilogue warps combine them and store Y.
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

constexpr int kSlices = kF64sSlices;   // S
constexpr int kSliceBits = 7;       // W
constexpr int kF64sM = 128;         // panel columns c per tile (TMEM lanes)
constexpr int kF64sN = 64;          // matrix rows n per tile
constexpr int kF64sSets = 1;        // accumulator sets in TMEM (7 groups x kF64sN columns each)
constexpr int kF64sKC = 32;         // K elements per stage (one 64-byte swizzle row of BF16)
constexpr int kF64sStages = 2;
constexpr int kF64sThreads = 640;   // warp 0: copies, warps 1-3: MMA, warps 4..19: epilogue
constexpr uint32_t kF64sPlaneA = kF64sM * 64;   // bytes of one panel plane per stage
constexpr uint32_t kF64sPlaneB = kF64sN * 64;   // bytes of one matrix plane per stage
constexpr uint32_t kF64sStageBytes = kSlices * (kF64sPlaneA + kF64sPlaneB);

// The 7 BF16 slices of v = x 2^-E (|v| < 1): the magnitude truncated to 49 bits, cut into
// 7-bit integers from the top, each carrying the sign of x.  Integer operations on the
// bits of x only.
__device__ __forceinline__ void slice7(double x, int E, uint16_t out[kSlices]) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int ebits = (int)((bits >> 52) & 0x7ff);
  const unsigned long long mant = (bits & 0xfffffffffffffull) | (ebits ? (1ull << 52) : 0ull);
  const int e_eff = ebits ? ebits : 1;
  // |x| = mant 2^(e_eff - 1075); F = |x| 2^(49 - E) = mant >> (1026 + E - e_eff)
  const int sh = 1026 + E - e_eff;
  const unsigned long long F = (sh >= 64 || sh < 0) ? 0ull : (mant >> sh);
  const uint16_t sign = (uint16_t)((bits >> 48) & 0x8000u);
#pragma unroll
  for (int i = 0; i < kSlices; ++i) {
    const uint32_t q = (uint32_t)(F >> (kSliceBits * (kSlices - 1 - i))) & ((1u << kSliceBits) - 1u);
    out[i] = (uint16_t)(__float_as_uint((float)q) >> 16) | (q ? sign : (uint16_t)0);
  }
}

// Exponent E with max|entries| < 2^E (0 for an all-zero vector).
__device__ __forceinline__ int exp_above(double m) {
  int e = 0;
  if (m > 0.0) frexp(m, &e);
  return e;
}

// Set-up: rows of every matrix (mats of Nr x Nr, row-major [n][j]) into 7 BF16 planes
// [mat * 7 + plane][n][pitch] and the row exponents rowexp[mat][n].  One warp per row.
__global__ void k_f64s_matrix(const double* __restrict__ A, int nmat, int Nr, int pitch, uint16_t* __restrict__ planes,
                              int32_t* __restrict__ rowexp) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= nmat * Nr) return;
  const int mat = warp / Nr, n = warp - mat * Nr;
  const double* row = A + ((size_t)mat * Nr + n) * Nr;
  double m = 0.0;
  for (int j = lane; j < Nr; j += 32) m = fmax(m, fabs(row[j]));
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int E = exp_above(m);
  if (lane == 0) rowexp[mat * Nr + n] = E;
  const size_t plane_elems = (size_t)Nr * pitch;
  for (int j = lane; j < pitch; j += 32) {
    uint16_t sl[kSlices];
    if (j < Nr) {
      slice7(row[j], E, sl);
    } else {
#pragma unroll
      for (int i = 0; i < kSlices; ++i) sl[i] = 0;
    }
#pragma unroll
    for (int i = 0; i < kSlices; ++i) planes[((size_t)mat * kSlices + i) * plane_elems + (size_t)n * pitch + j] = sl[i];
  }
}

// Per DHT: colmax[b][c] = max_j |X_b[j][c]| as the bits of a non-negative double (which
// order like the values), so that CTAs over slices of j combine with integer atomicMax;
// colmax starts at 0.  Grid: (columns / 256, rows / 32, items).
constexpr int kColRows = 32;
__global__ void k_f64s_colmax(DhtBatch bt, int Nr, int Nc, unsigned long long* __restrict__ colmax) {
  const int b = blockIdx.z;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= Nc) return;
  const double* X = static_cast<const double*>(bt.X[b]);
  const int j0 = blockIdx.y * kColRows, j1 = min(Nr, j0 + kColRows);
  // |x| as the bits with the sign cleared (non-negative doubles order like their bits):
  // integer compares, where fmax would run on the float64 unit
  unsigned long long m = 0ull;
#pragma unroll 8
  for (int j = j0; j < j1; ++j) {
    const unsigned long long a = (unsigned long long)__double_as_longlong(X[(size_t)j * Nc + c]) & 0x7fffffffffffffffull;
    m = a > m ? a : m;
  }
  if (m) atomicMax(colmax + (size_t)b * Nc + c, m);
}

// Per DHT: the panels into 7 K-major BF16 planes [b * 7 + plane][c][jpad].  Tiles of
// 64 columns x 32 rows j through shared memory: reads along c, writes along j.
constexpr int kPanelC = 64, kPanelJ = 32;
__global__ void __launch_bounds__(256) k_f64s_panel(DhtBatch bt, int Nr, int Nc, int jpad,
                                                    const unsigned long long* __restrict__ colmax,
                                                    int32_t* __restrict__ colexp, uint16_t* __restrict__ planes) {
  __shared__ __align__(16) uint16_t tile[kSlices][kPanelC][kPanelJ + 2];   // rows of 68 bytes
  const int b = blockIdx.z;
  const int c0 = blockIdx.x * kPanelC, j0 = blockIdx.y * kPanelJ;
  const double* X = static_cast<const double*>(bt.X[b]);
  const int tc = threadIdx.x & (kPanelC - 1), tj = threadIdx.x >> 6;   // 64 x 4
  const int c = c0 + tc;
  const int E = c < Nc ? exp_above(__longlong_as_double((long long)colmax[(size_t)b * Nc + c])) : 0;
  if (blockIdx.y == 0 && tj == 0 && c < Nc) colexp[(size_t)b * Nc + c] = E;   // for the epilogue
  double xv[kPanelJ / 4];   // all loads first, then the slicing
#pragma unroll
  for (int u = 0; u < kPanelJ / 4; ++u) {
    const int j = j0 + tj + 4 * u;
    xv[u] = (c < Nc && j < Nr) ? X[(size_t)j * Nc + c] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < kPanelJ / 4; ++u) {
    uint16_t sl[kSlices];
    slice7(xv[u], E, sl);
#pragma unroll
    for (int i = 0; i < kSlices; ++i) tile[i][tc][tj + 4 * u] = sl[i];
  }
  __syncthreads();
  // out: for each plane and column, kPanelJ consecutive j (64 bytes) as four 16-byte
  // stores of 8 j each (jpad and j0 are multiples of 8, so a group is inside the row or past
  // it whole; the tile's rows start on 4-byte boundaries: pitch 68 bytes)
  const size_t plane_elems = (size_t)Nc * jpad;
  constexpr int kQ = kPanelJ / 8;
  for (int idx = threadIdx.x; idx < kSlices * kPanelC * kQ; idx += blockDim.x) {
    const int i = idx / (kPanelC * kQ);
    const int rem = idx - i * kPanelC * kQ;
    const int cc = rem / kQ, jq = rem - cc * kQ;
    const int cg = c0 + cc, jg = j0 + 8 * jq;
    if (cg < Nc && jg < jpad) {
      const uint32_t* t32 = reinterpret_cast<const uint32_t*>(&tile[i][cc][8 * jq]);
      const uint4 v = make_uint4(t32[0], t32[1], t32[2], t32[3]);
      *reinterpret_cast<uint4*>(planes + ((size_t)b * kSlices + i) * plane_elems + (size_t)cg * jpad + jg) = v;
    }
  }
}

// SM100 shared-memory matrix descriptor: K-major, 64-byte swizzle (TMA's SWIZZLE_64B), 8-row
// groups 512 B apart.
__device__ __forceinline__ uint64_t make_desc_sw64(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);   // start address
  d |= (uint64_t)1u << 16;                   // leading byte offset (unused: K fits one row)
  d |= (uint64_t)(512u >> 4) << 32;          // stride byte offset: 8 rows x 64 B
  d |= (uint64_t)1u << 46;                   // descriptor version (SM100)
  d |= (uint64_t)4u << 61;                   // layout: SWIZZLE_64B
  return d;
}

// 3-D tiled tensor copy global -> shared (inner coordinate x, then y, z), completing its
// bytes on `bar`.  x is a multiple of 32 BF16 elements: 64-byte aligned.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tmap, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(tmap)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

struct F64sMaps {
  Sim::TensorMapBytes panel;   // [b * 7 + plane][c][j], box 32 j x 128 c
  Sim::TensorMapBytes mats;    // [mat * 7 + plane][n][j], box 32 j x 32 n
};

struct F64sParams {
  int Nr, Nc, n_tiles, m_tiles, tiles_total;
  int16_t mat[24];   // compact matrix index of each batch item
};

struct F64sTile {
  int b, n0, c0;
};

// n fastest: the CTAs that run at the same time share a panel tile (it stays in L2).
__device__ __forceinline__ F64sTile f64s_tile(int t, const F64sParams& P) {
  const int nt = t % P.n_tiles;
  const int rest = t / P.n_tiles;
  return F64sTile{rest / P.m_tiles, nt * kF64sN, (rest % P.m_tiles) * kF64sM};
}

__global__ void __launch_bounds__(kF64sThreads, 1) k_dht_f64s(DhtBatch bt, F64sParams P,
                                                               const __grid_constant__ F64sMaps maps,
                                                               const int32_t* __restrict__ colexp,
                                                               const int32_t* __restrict__ rowexp, int32_t* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(base + kF64sStages * kF64sStageBytes);
  uint64_t* empty = full + kF64sStages;
  uint64_t* tfull = empty + kF64sStages;
  uint64_t* tempty = tfull + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nK = (P.Nr + kF64sKC - 1) / kF64sKC;
  constexpr uint32_t kTmemCols = 512;                 // sets x 7 groups x kF64sN columns <= 512
  constexpr uint32_t kSetCols = kSlices * kF64sN;

  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    for (int i = 0; i < kF64sStages; ++i) {
      mbar_init(&full[i], 1);    // the copy issuer's arrive.expect_tx
      mbar_init(&empty[i], 3);   // one MMA commit per issuing warp
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 3);   // the issuing warps' commits after a tile's last chunk
      mbar_init(&tempty[i], 16);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;
  // kind::f16: D f32, A and B bf16, both K-major; N = 32, M = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kF64sN >> 3) << 17) |
                         ((uint32_t)(kF64sM >> 4) << 24);

  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(err, kErrTimeout);
  };

  if (warp == 0) {
    // ---------------------------------------------------------------- copy issuer
    if (lane == 0) {
      uint32_t g = 0;
      int last_armed = -1;
      for (int t = blockIdx.x; t < P.tiles_total && !*abort_flag; t += gridDim.x) {
        const F64sTile w = f64s_tile(t, P);
        const int zm = P.mat[w.b] * kSlices, zp = w.b * kSlices;
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int st = (int)(g % (uint32_t)kF64sStages);
          const uint32_t use = g / (uint32_t)kF64sStages;
          if (use > 0 && !mbar_wait(&empty[st], (use - 1) & 1)) { fail(); ok = false; break; }
          if (*abort_flag) { ok = false; break; }
          unsigned char* sA = base + st * kF64sStageBytes;
          unsigned char* sB = sA + kSlices * kF64sPlaneA;
          mbar_arrive_expect_tx(&full[st], kF64sStageBytes);
#pragma unroll
          for (int p = 0; p < kSlices; ++p)
            tma_load_3d(sA + p * kF64sPlaneA, &maps.panel, kc * kF64sKC, w.c0, zp + p, &full[st]);
#pragma unroll
          for (int p = 0; p < kSlices; ++p)
            tma_load_3d(sB + p * kF64sPlaneB, &maps.mats, kc * kF64sKC, w.n0, zm + p, &full[st]);
          last_armed = st;
        }
        if (!ok) break;
      }
      // before shared memory is released: the last armed stage's copies must have landed
      if (last_armed >= 0 && *abort_flag) {
        const uint32_t gl = g == 0 ? 0 : g - 1;
        mbar_wait(&full[last_armed], (gl / (uint32_t)kF64sStages) & 1);
      }
    }
    __syncwarp();
  } else if (warp >= 1 && warp <= 3) {
    // ---------------------------------------------------------------- MMA issuers
    // Three warps issue the products, each into its own accumulator groups (so every
    // group's first, overwriting product comes from one thread): warp 1 groups 0, 1, 6 (10
    // products per 16 K), warp 2 groups 2, 5 (9), warp 3 groups 3, 4 (9).  One thread
    // issuing all 28 left the tensor pipe three quarters idle.
    if (lane == 0) {
      const uint32_t gmask = warp == 1 ? 0x43u : (warp == 2 ? 0x24u : 0x18u);   // groups of this warp
      uint32_t g = 0, i = 0;
      uint64_t* last_bar = nullptr;
      uint32_t last_parity = 0;
      for (int t = blockIdx.x; t < P.tiles_total && !*abort_flag; t += gridDim.x, ++i) {
        const uint32_t set = i % kF64sSets, set_use = i / kF64sSets;
        if (set_use > 0 && !mbar_wait(&tempty[set], (set_use - 1) & 1)) { fail(); break; }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d0 = tmem + set * kSetCols;
        bool ok = true;
        for (int kc = 0; kc < nK; ++kc, ++g) {
          const int st = (int)(g % (uint32_t)kF64sStages);
          if (!mbar_wait(&full[st], (g / (uint32_t)kF64sStages) & 1)) { fail(); ok = false; break; }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t sa = smem_u32(base + st * kF64sStageBytes), sb = sa + kSlices * kF64sPlaneA;
#pragma unroll
          for (int ks = 0; ks < 2; ++ks) {
            const uint32_t koff = ks * 32;
#pragma unroll
            for (int grp = 0; grp < kSlices; ++grp) {
              if (!((gmask >> grp) & 1u)) continue;
#pragma unroll
              for (int ia = 0; ia <= grp; ++ia) {   // matrix slice ia, panel slice grp - ia
                const uint32_t accf = (kc > 0 || ks > 0 || ia > 0) ? 1u : 0u;
                mma_f16(d0 + grp * kF64sN, make_desc_sw64(sa + (grp - ia) * kF64sPlaneA + koff),
                        make_desc_sw64(sb + ia * kF64sPlaneB + koff), idesc, accf);
              }
            }
          }
          mma_commit(&empty[st]);
          last_bar = &empty[st];
          last_parity = (g / (uint32_t)kF64sStages) & 1;
        }
        if (!ok) break;
        mma_commit(&tfull[set]);
        last_bar = &tfull[set];
        last_parity = (i / kF64sSets) & 1;
      }
      if (*abort_flag && last_bar) mbar_wait(last_bar, last_parity);
    }
    __syncwarp();
  } else if (warp >= 4) {
    // ---------------------------------------------------------------- epilogue (warps 4-19)
    // four warps per TMEM lane quarter (warp % 4 == q: lanes 32q .. 32q + 31), each taking
    // a quarter of the tile's columns
    const int q = warp & 3, jh = ((warp - 4) >> 2) * (kF64sN / 4);
    uint32_t i = 0;
    for (int t = blockIdx.x; t < P.tiles_total && !*abort_flag; t += gridDim.x, ++i) {
      const uint32_t set = i % kF64sSets;
      if (!mbar_wait(&tfull[set], (i / kF64sSets) & 1)) { fail(); break; }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const F64sTile w = f64s_tile(t, P);
      double* __restrict__ Y = static_cast<double*>(bt.Y[w.b]);
      const int c = w.c0 + q * 32 + lane;
      const int Ec = c < P.Nc ? colexp[(size_t)w.b * P.Nc + c] : 0;
      const int32_t* rexp = rowexp + (size_t)P.mat[w.b] * P.Nr;
      for (int j0 = jh; j0 < jh + kF64sN / 4; j0 += 8) {
        // the group sums of 8 columns: groups 0..3 exact integers below 2^24 in float,
        // groups 4..6 below 2^25 within one rounding
        uint32_t r[kSlices][8];
#pragma unroll
        for (int grp = 0; grp < kSlices; ++grp) {
          const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + set * kSetCols + grp * kF64sN + (uint32_t)j0;
          asm volatile(
              "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
              : "=r"(r[grp][0]), "=r"(r[grp][1]), "=r"(r[grp][2]), "=r"(r[grp][3]), "=r"(r[grp][4]),
                "=r"(r[grp][5]), "=r"(r[grp][6]), "=r"(r[grp][7])
              : "r"(taddr)
              : "memory");
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c < P.Nc) {
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            const int n = w.n0 + j0 + e;
            if (n >= P.Nr) continue;
            // sum_g acc_g 2^(-7(g+2)) = T 2^-49 with
            //   T = (((a0 2^7 + a1) 2^7 + a2) 2^7 + a3) 2^14 + a4 2^7 + a5 + round(a6 2^-7),
            // all in integer arithmetic: a0..a3 are exact integers below 2^24, a4..a6
            // integer-valued floats below 2^25 (their sums were rounded at weight <= 2^-42);
            // |T| < 2^58.  Then one int -> double conversion, the only float64 instruction
            // (GB300's float64 unit is the scarce one), and the scaling by 2^k as an addition
            // to the exponent field while the result stays normal.
            const long long a0 = __float2int_rn(__uint_as_float(r[0][e]));
            const long long a1 = __float2int_rn(__uint_as_float(r[1][e]));
            const long long a2 = __float2int_rn(__uint_as_float(r[2][e]));
            const long long a3 = __float2int_rn(__uint_as_float(r[3][e]));
            const long long a4 = __float2int_rn(__uint_as_float(r[4][e]));
            const long long a5 = __float2int_rn(__uint_as_float(r[5][e]));
            const long long a6 = __float2int_rn(__uint_as_float(r[6][e]) * (1.f / 128.f));
            const long long T = (((a0 * 128 + a1) * 128 + a2) * 128 + a3) * 16384 + a4 * 128 + a5 + a6;
            const int k = Ec + rexp[n] - kSliceBits * kSlices;   // 2^(E_c + E_n - 49)
            const double t = (double)T;
            long long bits = __double_as_longlong(t);
            const int ex = (int)((bits >> 52) & 0x7ff) + k;
            double y;
            if (T != 0 && ex > 0 && ex < 2047) {
              bits += (long long)k * (1LL << 52);
              y = __longlong_as_double(bits);
            } else {
              y = t * ldexp(1.0, k);   // zero, or a result outside the normal range
            }
            Y[(size_t)n * P.Nc + c] = y;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[set]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (warp == 1)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

constexpr size_t kF64sSmem = 1024 + (size_t)kF64sStages * kF64sStageBytes + 256;
static_assert(kF64sSets * kSlices * kF64sN <= 512, "accumulators exceed tensor memory");
static_assert(kF64sSmem <= 227 * 1024, "stages exceed shared memory");

int f64s_pitch(int Nr) { return split_pitch_b16(Nr); }   // BF16 row pitch, 16-byte rows

int blocks_for(size_t n, int t) { return (int)((n + t - 1) / t); }

}  // namespace

bool f64s_supported(const pic_config& c) { return c.precision == PIC_FP64 && c.Nr <= kF64sMaxNr; }

bool f64s_active(const Sim* s) { return f64s_supported(s->cfg) && s->dht_path != PIC_DHT_F64_GEMM; }

pic_status f64s_configure_device() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PIC_OK;
  PIC_CUDA(cudaFuncSetAttribute(k_dht_f64s, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kF64sSmem));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

// Set-up (after the FP64 matrices are final): slices of the forward matrices (compact
// index 0 .. 3Nm-1) and of the inverse matrices (3Nm .. 6Nm-1).
pic_status launch_f64s_setup(Sim* s) {
  if (!f64s_supported(s->cfg)) return PIC_OK;
  const int Nr = s->cfg.Nr, nm3 = 3 * s->cfg.Nm, pitch = f64s_pitch(Nr);
  uint16_t* planes = s->at<uint16_t>(s->lay.f64s_mat);
  int32_t* rowexp = s->at<int32_t>(s->lay.f64s_rowexp);
  const size_t mat_elems = (size_t)kSlices * Nr * pitch;
  const int blocks = blocks_for((size_t)nm3 * Nr * 32, 256);
  k_f64s_matrix<<<blocks, 256, 0, s->stream>>>(s->at<double>(s->lay.mfwd), nm3, Nr, pitch, planes, rowexp);
  PIC_LAUNCHED(s);
  k_f64s_matrix<<<blocks, 256, 0, s->stream>>>(s->at<double>(s->lay.binv), nm3, Nr, pitch,
                                               planes + (size_t)nm3 * mat_elems, rowexp + (size_t)nm3 * Nr);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

// Tensor maps of the panel planes and matrix planes (3-D: inner j, then c or n, then
// item or matrix x plane), 64-byte swizzle; coordinates past Nr (j, n) or Nc read zero.
pic_status f64s_make_maps(Sim* s) {
  std::memset(s->f64s_maps, 0, sizeof(s->f64s_maps));
  if (!f64s_supported(s->cfg)) return PIC_OK;
  using Encode = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
  Encode encode = reinterpret_cast<Encode>(tensor_map_encoder());
  if (!encode) {
    set_error("cuTensorMapEncodeTiled is not available from the driver");
    return PIC_ERR_CUDA;
  }
  const int Nr = s->cfg.Nr, Nc = 2 * s->cfg.Nz, pitch = f64s_pitch(Nr);
  const cuuint32_t estr[3] = {1, 1, 1};
  {
    const cuuint64_t dims[3] = {(cuuint64_t)Nr, (cuuint64_t)Nc, (cuuint64_t)(6 * s->cfg.Nm * kSlices)};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)Nc * pitch * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kF64sKC, (cuuint32_t)kF64sM, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(s->f64s_maps[0].b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                              s->at<char>(s->lay.f64s_panel), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled failed (%d) for the sliced panels", (int)r);
      return PIC_ERR_CUDA;
    }
  }
  {
    const cuuint64_t dims[3] = {(cuuint64_t)Nr, (cuuint64_t)Nr, (cuuint64_t)(6 * s->cfg.Nm * kSlices)};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * 2, (cuuint64_t)Nr * pitch * 2};
    const cuuint32_t box[3] = {(cuuint32_t)kF64sKC, (cuuint32_t)kF64sN, 1};
    const CUresult r = encode(reinterpret_cast<CUtensorMap*>(s->f64s_maps[1].b), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3,
                              s->at<char>(s->lay.f64s_mat), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                              CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) {
      set_error("cuTensorMapEncodeTiled failed (%d) for the sliced matrices", (int)r);
      return PIC_ERR_CUDA;
    }
  }
  return PIC_OK;
}

// Y = A X of a batch in the FP64 form on the tensor cores: column exponents, panel slices,
// then the persistent product kernel.
pic_status launch_dht_f64s(Sim* s, const DhtBatch& b) {
  const int Nr = s->cfg.Nr, Nc = 2 * s->cfg.Nz, Nm = s->cfg.Nm, pitch = f64s_pitch(Nr);
  if (b.n < 1 || b.n > 6 * Nm) {
    set_error("sliced FP64 DHT: batch of %d items (1 .. %d)", b.n, 6 * Nm);
    return PIC_ERR_ARG;
  }
  F64sParams P{};
  P.Nr = Nr;
  P.Nc = Nc;
  P.n_tiles = (Nr + kF64sN - 1) / kF64sN;
  P.m_tiles = (Nc + kF64sM - 1) / kF64sM;
  P.tiles_total = P.n_tiles * P.m_tiles * b.n;
  for (int i = 0; i < b.n; ++i) {
    const int id = b.mat[i], per = kMaxModes * 3;
    const int dir = id / per, mi = id % per;
    if (id < 0 || dir > 1 || mi >= 3 * Nm) {
      set_error("sliced FP64 DHT: batch entry %d has no matrix", i);
      return PIC_ERR_ARG;
    }
    P.mat[i] = (int16_t)(dir * 3 * Nm + mi);
  }
  int32_t* colexp = s->at<int32_t>(s->lay.f64s_colexp);
  unsigned long long* colmax = reinterpret_cast<unsigned long long*>(colexp + (size_t)6 * Nm * Nc);
  PIC_CUDA(cudaMemsetAsync(colmax, 0, (size_t)b.n * Nc * sizeof(unsigned long long), s->stream));
  k_f64s_colmax<<<dim3(blocks_for(Nc, 256), blocks_for(Nr, kColRows), b.n), 256, 0, s->stream>>>(b, Nr, Nc, colmax);
  PIC_LAUNCHED(s);
  k_f64s_panel<<<dim3(blocks_for(Nc, kPanelC), blocks_for(Nr, kPanelJ), b.n), 256, 0, s->stream>>>(
      b, Nr, Nc, pitch, colmax, colexp, s->at<uint16_t>(s->lay.f64s_panel));
  PIC_LAUNCHED(s);
  F64sMaps maps;
  maps.panel = s->f64s_maps[0];
  maps.mats = s->f64s_maps[1];
  const int grid = std::min(P.tiles_total, dht_tc_sm_count());
  k_dht_f64s<<<grid, kF64sThreads, kF64sSmem, s->stream>>>(b, P, maps, colexp, s->at<int32_t>(s->lay.f64s_rowexp),
                                                           s->at<int32_t>(s->lay.err));
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
