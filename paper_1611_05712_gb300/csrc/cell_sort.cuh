// Sorting the particle indices of one crowded cell (part of the stable counting sort by
// cell key: after the scatter, the indices of a cell sit in arbitrary order and are put
// back in ascending order, which makes the sort stable and deterministic).
//
// Two routines with bounded cost per cell:
//   warp_rank_cell  one warp, each entry ranked against all others: for the cells of a
//                   moderate count (<= kWarpCellMax entries, at most kWarpCellMax^2 / 32
//                   comparisons per lane);
//   cta_sort_cell   one CTA: bitonic sort of chunks of kCellChunk entries in shared
//                   memory, then merge passes of doubling width between two global
//                   buffers (each pass splits the outputs among the threads by a binary
//                   search along the merge path).  O(n log n) work for any count, so a
//                   cell holding every particle costs a few passes over its entries.
#pragma once

#include <stdint.h>

namespace pic {

constexpr int kWarpCellMax = 128;
constexpr int kCellChunk = 2048;   // shared-memory chunk of cta_sort_cell (8 KB)

// out[rank] = entry, rank = number of smaller entries; entries are distinct indices.
__device__ __forceinline__ void warp_rank_cell(const int32_t* in, int32_t* out, int n) {
  const int lane = threadIdx.x & 31;
  for (int k = lane; k < n; k += 32) {
    const int32_t e = in[k];
    int rank = 0;
    for (int q = 0; q < n; ++q) rank += (in[q] < e);
    out[rank] = e;
  }
}

// Sorts the n distinct values in[0..n) ascending into out[0..n), using alt[0..n) as the
// second buffer of the merge passes.  alt may be the same memory as in (in is fully read
// before the first merge pass).  Called by every thread of the CTA, with sm holding
// kCellChunk int32 of shared memory.  Ends with the CTA synchronised.
__device__ __forceinline__ void cta_sort_cell(const int32_t* in, int32_t* out, int32_t* alt, int n,
                                              int32_t* sm) {
  const int tid = threadIdx.x, nt = blockDim.x;
  // phase 1: sorted runs of kCellChunk
  for (int b = 0; b < n; b += kCellChunk) {
    const int cnt = min(kCellChunk, n - b);
    int P = 1;
    while (P < cnt) P <<= 1;
    for (int i = tid; i < P; i += nt) sm[i] = i < cnt ? in[b + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1) {
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int i = tid; i < P; i += nt) {
          const int l = i ^ j;
          if (l > i) {
            const int32_t a = sm[i], c = sm[l];
            if ((a > c) == ((i & k) == 0)) { sm[i] = c; sm[l] = a; }
          }
        }
        __syncthreads();
      }
    }
    for (int i = tid; i < cnt; i += nt) out[b + i] = sm[i];
    __syncthreads();
  }
  if (n <= kCellChunk) return;
  // phase 2: merge pairs of runs, ping-ponging between out and alt
  constexpr int E = 8;   // outputs per thread and step
  int32_t* src = out;
  int32_t* dst = alt;
  for (int w = kCellChunk; w < n; w <<= 1) {
    for (int k0 = tid * E; k0 < n; k0 += nt * E) {
      const int a0 = k0 / (2 * w) * (2 * w);
      const int lenA = min(w, n - a0);
      const int lenB = max(0, min(w, n - a0 - w));
      const int32_t* A = src + a0;
      const int32_t* B = A + lenA;
      const int k = k0 - a0;
      int lo = max(0, k - lenB), hi = min(k, lenA);
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (A[mid] < B[k - mid - 1]) lo = mid + 1; else hi = mid;
      }
      int i = lo, j = k - lo;
      const int kend = min(k + E, lenA + lenB);
      for (int q = k; q < kend; ++q) {
        int32_t v;
        if (j >= lenB || (i < lenA && A[i] < B[j])) v = A[i++]; else v = B[j++];
        dst[a0 + q] = v;
      }
    }
    __syncthreads();
    int32_t* t = src; src = dst; dst = t;
  }
  if (src != out) {
    for (int i = tid; i < n; i += nt) out[i] = src[i];
    __syncthreads();
  }
}

}  // namespace pic
