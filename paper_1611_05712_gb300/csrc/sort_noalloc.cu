// Allocation-free cell-key sort: pic_sort_keys_noalloc (declared in include/psatd_rz.h).
//
// Some callers cannot allocate device memory at the moment they need the sort:
// applications that hand this library a fixed memory budget at start-up and forbid any
// allocation afterwards, or hosts whose own allocator owns the whole device and keeps
// cudaMalloc out of reach of the libraries they load.  This entry point needs no
// workspace from them: its scratch (per-cell counts, offsets, scatter cursors, the
// unsorted index list, the queue of crowded cells) lives in one file-scope __device__
// array of fixed size, which every GPU that loads the library holds until the process
// exits.
//
// It computes the cell keys and the stable permutation of the sort stage of the FP64
// PIC cycle without a moving window (pic_sort on a PIC_FP64 handle), with kernels of its
// own; the ordering of crowded cells shares cell_sort.cuh with pic_sort.
#include <mutex>

#include "cell_sort.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kNaMaxCells = 65536;          // Nz * Nr
constexpr int kNaMaxParticles = 262144;
constexpr int kNaMaxHuge = kNaMaxParticles / (kWarpCellMax + 1) + 1;   // cells sorted by a CTA
constexpr int kNaMaxDevices = 64;
// int32 layout: count[cells + 1] | start[cells + 1] | cursor[cells] | tmp[particles] |
// nhuge[1] | huge[kNaMaxHuge]
constexpr size_t kNaCount = 0;
constexpr size_t kNaStart = kNaCount + kNaMaxCells + 1;
constexpr size_t kNaCursor = kNaStart + kNaMaxCells + 1;
constexpr size_t kNaTmp = kNaCursor + kNaMaxCells;
constexpr size_t kNaNHuge = kNaTmp + kNaMaxParticles;
constexpr size_t kNaHuge = kNaNHuge + 1;
constexpr size_t kNaInts = kNaHuge + kNaMaxHuge;   // 1.84 MB

static __device__ __align__(256) int32_t g_sort_scratch[kNaInts];

__global__ void k_na_zero(int32_t* sc, int ncell) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= ncell; i += gridDim.x * blockDim.x)
    sc[kNaCount + i] = 0;
  if (blockIdx.x == 0 && threadIdx.x == 0) sc[kNaNHuge] = 0;
}

__global__ void k_na_keys(const double* x, const double* y, const double* z, int n, int Nz, int Nr,
                          double dz, double dr, int32_t* keys, int32_t* sc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double xi = x[i], yi = y[i];
    const double r = sqrt(__dadd_rn(__dmul_rn(xi, xi), __dmul_rn(yi, yi)));
    double fz = floor(z[i] / dz), fr = floor(r / dr);
    if (!(fz == fz) || isinf(fz)) fz = 0.0;   // non-finite coordinates go to cell 0
    if (!(fr == fr) || isinf(fr)) fr = 0.0;
    const int iz = (int)fmin(fmax(fz, 0.0), (double)(Nz - 1));
    const int ir = (int)fmin(fmax(fr, 0.0), (double)(Nr - 1));
    const int key = iz * Nr + ir;
    keys[i] = key;
    atomicAdd(sc + kNaCount + key, 1);
  }
}

// One block: exclusive scan of count[0..ncell) into start (and cursor); start[ncell] = n.
__global__ void __launch_bounds__(1024) k_na_scan(int32_t* sc, int ncell) {
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < ncell; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int32_t v = i < ncell ? sc[kNaCount + i] : 0;
    int32_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += t;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    if (warp == 0) {
      int32_t t = warp_tot[lane];
      for (int o = 1; o < 32; o <<= 1) {
        const int32_t u = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += u;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const int32_t excl = carry + x - v + (warp > 0 ? warp_tot[warp - 1] : 0);
    if (i < ncell) {
      sc[kNaStart + i] = excl;
      sc[kNaCursor + i] = excl;
    }
    __syncthreads();
    if (threadIdx.x == 0) carry += warp_tot[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) sc[kNaStart + ncell] = carry;
}

__global__ void k_na_scatter(const int32_t* keys, int n, int32_t* sc) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int32_t pos = atomicAdd(sc + kNaCursor + keys[i], 1);
    sc[kNaTmp + pos] = i;
  }
}

// One warp per cell: the indices of a cell, ranked ascending, give the stable order.
// Cells of more than kWarpCellMax entries are queued for k_na_cell_big.
__global__ void k_na_cell_rank(int32_t* sc, int ncell, int32_t* perm) {
  const int nw = (gridDim.x * blockDim.x) >> 5;
  for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncell; c += nw) {
    const int s0 = sc[kNaStart + c], cnt = sc[kNaStart + c + 1] - s0;
    if (cnt <= kWarpCellMax) {
      warp_rank_cell(sc + kNaTmp + s0, perm + s0, cnt);
    } else if ((threadIdx.x & 31) == 0) {
      sc[kNaHuge + atomicAdd(sc + kNaNHuge, 1)] = c;
    }
  }
}

// One CTA per queued cell: O(n log n) ordering (cell_sort.cuh), the cell's range of the
// index list serving as the second buffer.
__global__ void __launch_bounds__(256) k_na_cell_big(int32_t* sc, int32_t* perm) {
  __shared__ int32_t sm[kCellChunk];
  const int nh = sc[kNaNHuge];
  for (int b = blockIdx.x; b < nh; b += gridDim.x) {
    const int c = sc[kNaHuge + b];
    const int s0 = sc[kNaStart + c], cnt = sc[kNaStart + c + 1] - s0;
    int32_t* t = sc + kNaTmp + s0;
    cta_sort_cell(t, perm + s0, t, cnt, sm);
  }
}

std::mutex g_na_mutex;
int32_t* g_na_ptr[kNaMaxDevices] = {};

// Device address of the scratch array for the current device (looked up once per device).
pic_status na_scratch(int32_t** out) {
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return PIC_ERR_ARG;
  }
  std::lock_guard<std::mutex> lock(g_na_mutex);
  if (!g_na_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_sort_scratch);
    if (e != cudaSuccess) return cuda_status(e, "cudaGetSymbolAddress(g_sort_scratch)");
    g_na_ptr[dev] = static_cast<int32_t*>(p);
  }
  *out = g_na_ptr[dev];
  return PIC_OK;
}

}  // namespace
}  // namespace pic

using namespace pic;

extern "C" pic_status pic_sort_keys_noalloc(const double* x, const double* y, const double* z, int64_t n,
                                            int32_t Nz, int32_t Nr, double dz, double dr, int32_t* keys,
                                            int32_t* perm, void* stream) {
  if (n < 0 || n > kNaMaxParticles) {
    set_error("pic_sort_keys_noalloc: n=%lld outside [0, %d]", (long long)n, kNaMaxParticles);
    return PIC_ERR_ARG;
  }
  if (Nz < 1 || Nr < 1 || (int64_t)Nz * Nr > kNaMaxCells) {
    set_error("pic_sort_keys_noalloc: Nz*Nr=%lld outside [1, %d]", (long long)Nz * Nr, kNaMaxCells);
    return PIC_ERR_ARG;
  }
  if (!(dz > 0) || !(dr > 0)) { set_error("pic_sort_keys_noalloc: dz, dr must be > 0"); return PIC_ERR_ARG; }
  if (n > 0 && (!x || !y || !z || !keys || !perm)) {
    set_error("pic_sort_keys_noalloc: NULL pointer");
    return PIC_ERR_ARG;
  }
  int32_t* sc = nullptr;
  pic_status st = na_scratch(&sc);
  if (st != PIC_OK) return st;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int ncell = Nz * Nr;
  const int ni = (int)n;
  k_na_zero<<<(ncell + 256) / 256, 256, 0, s>>>(sc, ncell);
  PIC_CUDA(cudaGetLastError());
  if (ni > 0) {
    const int pb = (ni + 255) / 256 < 1216 ? (ni + 255) / 256 : 1216;
    k_na_keys<<<pb, 256, 0, s>>>(x, y, z, ni, Nz, Nr, dz, dr, keys, sc);
    PIC_CUDA(cudaGetLastError());
    k_na_scan<<<1, 1024, 0, s>>>(sc, ncell);
    PIC_CUDA(cudaGetLastError());
    k_na_scatter<<<pb, 256, 0, s>>>(keys, ni, sc);
    PIC_CUDA(cudaGetLastError());
    const int cb = (ncell * 32 + 255) / 256 < 2432 ? (ncell * 32 + 255) / 256 : 2432;
    k_na_cell_rank<<<cb, 256, 0, s>>>(sc, ncell, perm);
    PIC_CUDA(cudaGetLastError());
    k_na_cell_big<<<152, 256, 0, s>>>(sc, perm);
    PIC_CUDA(cudaGetLastError());
  }
  return PIC_OK;
}
