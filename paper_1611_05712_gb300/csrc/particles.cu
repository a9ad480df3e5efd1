// Particle stages of the PIC cycle (the PIC loop of the introduction; deposition,
// gather and push are the particle side of the quasi-cylindrical scheme of section
// "Finite order pseudo-spectral solvers"):
//   a1 cell keys + stable counting sort, a2 gather with mode reconstruction,
//   a3 relativistic Boris push, a4 charge / current deposition per mode,
//   a10 FP64 beam diagnostics (emittance, slice energy spread; section "Accurate
//   modeling of plasma accelerators in finite order PSATD").
// Conventions: F = Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}], deposit weight e^{+i m theta},
// linear weights in z (periodic) and r (nodes r_j = (j+1/2) dr), ghost node j = -1
// folded into node 0 with sign (-1)^m (scalar, z) or (-1)^{m+1} (r, theta), node Nr
// dropped, cell volume 2 pi r_j dr dz.
#include <math.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "cell_sort.cuh"
#include "dword.cuh"
#include "pic_internal.cuh"

namespace pic {
namespace {

struct Parts {
  double* x; double* y; double* z; double* ux; double* uy; double* uz; double* w;
  int32_t* id;
};

Parts parts_of(Sim* s, int which) {
  Parts p;
  double** a = &p.x;
  for (int k = 0; k < 7; ++k) a[k] = s->at<double>(s->lay.part[which][k]);
  p.id = s->at<int32_t>(s->lay.pid[which]);
  return p;
}

struct GridGeom {
  int Nz, Nr, Nm;
  double dz, dr, L, R;
  size_t G;      // Nm*Nr*Nz
  double inv_dr; // 1/dr, 1/dz correctly rounded (float64 divisions are long sequences on
  double inv_dz; // GB300's float64 unit)
};

GridGeom geom_of(const Sim* s) {
  const pic_config& c = s->cfg;
  GridGeom g{c.Nz, c.Nr, c.Nm, c.dz, c.dr, c.Nz * c.dz, c.Nr * c.dr, s->grid_elems(), 1.0 / c.dr, 1.0 / c.dz};
  return g;
}

constexpr double kInvC2 = 1.0 / (kC * kC);   // gamma from u without a float64 division

// r, cos(theta), sin(theta) of (x, y) from one reciprocal square root (CUDA's rsqrt, within
// one ulp): with q = x^2 + y^2, r = q rsqrt(q) and (cos, sin) = (x, y) rsqrt(q), within about
// two ulps, without a square root and a division.  The axis (q = 0) takes theta = 0.
__device__ __forceinline__ void polar(double x, double y, double& r, double& c, double& s) {
  const double r2 = __dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y));
  if (r2 > 0.0) {
    const double ir = rsqrt(r2);
    r = r2 * ir; c = x * ir; s = y * ir;
  } else {
    r = 0.0; c = 1.0; s = 0.0;
  }
}

struct Stencil {
  int i0, i1, j0;
  double wz0, wz1, wr0, wr1;
};

// x / d correctly rounded without a division, from inv_d = the correctly rounded 1/d: q =
// x inv_d, then twice q <- q + (x - q d) inv_d, the remainder exact in one fma; the first
// correction makes q a faithful quotient and the second returns the correctly rounded one
// (Markstein, IBM J. Res. Dev. 34, 1990).  An infinite or NaN x gives NaN.
__device__ __forceinline__ double div_rn(double x, double d, double inv_d) {
  double q = __dmul_rn(x, inv_d);
  q = __fma_rn(__fma_rn(-q, d, x), inv_d, q);
  return __fma_rn(__fma_rn(-q, d, x), inv_d, q);
}

__device__ __forceinline__ Stencil stencil(const GridGeom& g, double z, double r) {
  Stencil st;
  double u = div_rn(z, g.dz, g.inv_dz);
  double fi = floor(u);
  double sz = u - fi;
  long long i0 = (long long)fi;
  if (i0 < 0 || i0 >= g.Nz) {   // z outside [0, L): wrap (the push keeps z inside)
    i0 %= g.Nz;
    if (i0 < 0) i0 += g.Nz;
  }
  st.i0 = (int)i0;
  st.i1 = st.i0 + 1 == g.Nz ? 0 : st.i0 + 1;
  st.wz0 = 1.0 - sz;
  st.wz1 = sz;
  // z / dz stays correctly rounded (one ulp of it is ~Nz ulps of a weight); r / dr (r < R)
  // as a product with 1/dr
  double v = r * g.inv_dr - 0.5;
  double fj = floor(v);
  double t = v - fj;
  // r >= 0 gives fj >= -1; beyond the last node every weight is dropped anyway
  st.j0 = (int)fmin(fmax(fj, -1.0), (double)g.Nr);
  st.wr0 = 1.0 - t;
  st.wr1 = t;
  return st;
}

// Gather weights of a particle's 4 nodes n = 2 dz + dj (rows i0, i1; radial nodes j0, j0 + 1):
// w_z w_r, 0 for a dropped node (j >= Nr, read at a valid address); the ghost node r = -dr/2
// of the axis cell (j0 = -1) is read at node 0 and takes its field's fold sign.
struct GatherNodes {
  double w[4];
  size_t off[4];   // j Nz + i
  bool ghost;
};

__device__ __forceinline__ GatherNodes gather_nodes(const GridGeom& g, const Stencil& st) {
  GatherNodes gn;
#pragma unroll
  for (int n = 0; n < 4; ++n) {
    const int dz = n >> 1, dj = n & 1;
    const int j = st.j0 + dj;
    const bool keep = j < g.Nr;
    const int jj = (j < 0 || !keep) ? 0 : j;
    gn.w[n] = keep ? (dz ? st.wz1 : st.wz0) * (dj ? st.wr1 : st.wr0) : 0.0;
    gn.off[n] = (size_t)jj * g.Nz + (dz ? st.i1 : st.i0);
  }
  gn.ghost = st.j0 < 0;
  return gn;
}

// Gather in double words (FP64 form): the mode sum of the gather above with every product
// and sum on the float32 units, from the double-word copy of E, B that the inverse row FFT
// writes ([6][Nm][Nr][Nz] float4: re.hi, re.lo, im.hi, im.lo).  Each component is one dot
// product of double words, accumulated after Ogita, Rump and Oishi's Dot2 (SIAM J. Sci.
// Comput. 26, 2005): the products of the high parts enter a float sum through an
// error-free two-sum, whose errors, with each product's rounding error (one fma) and its
// cross terms, collect in a second float.  The error stays below a few 2^-48 times the sum
// of the terms' magnitudes (n u^2 for the n = 8 Nm - 4 terms of a component, u = 2^-24,
// plus the operands' own double-word rounding), against the n 2^-53 of a float64 sum;
// GB300 runs float64 at 1/64 of its float32 rate, and the float64 unit bounds the particle
// pass.
struct Dot2 {
  float s, c;   // running sum and collected errors: the value is s + c
};

__device__ __forceinline__ void dot2_add(Dot2& a, dw x, float yh, float yl) {
  const float p = __fmul_rn(x.hi, yh);
  const float e = __fmaf_rn(x.hi, yh, -p);   // p + e = x.hi yh exactly
  const float t = __fadd_rn(a.s, p);         // two-sum: t + err = s + p exactly
  const float bb = __fsub_rn(t, a.s);
  const float err = __fadd_rn(__fsub_rn(a.s, __fsub_rn(t, bb)), __fsub_rn(p, bb));
  a.s = t;
  a.c = __fadd_rn(a.c, __fadd_rn(err, __fmaf_rn(x.hi, yl, __fmaf_rn(x.lo, yh, e))));
}

__device__ __forceinline__ dw dw_twice(dw x) { return dw(__fmul_rn(2.f, x.hi), __fmul_rn(2.f, x.lo)); }

// F_k = Re sum_m mult_m e^{-i m theta} sum_n w_n F_{k,m}(node n) as in k_gather_push, with
// 2 Re(e^{-i m theta} v) = 2 cos(m theta) Re v + 2 sin(m theta) Im v; the inner nodes (n = 0,
// 2) take their field's fold sign through sign-flipped copies of their weights.
__device__ __forceinline__ void gather_dw(const GridGeom& g, const GatherNodes& gn, double c, double s,
                                          const float4* __restrict__ EB, double (&F)[6]) {
  const size_t RZ = (size_t)g.Nr * g.Nz;
  dw w[4];
#pragma unroll
  for (int n = 0; n < 4; ++n) w[n] = dw_from_double(gn.w[n]);
  Dot2 acc[6];
  {   // mode 0: real part; fold +1 for z components, -1 for r and theta
    const dw f0 = neg_if(w[0], gn.ghost), f2 = neg_if(w[2], gn.ghost);
#pragma unroll
    for (int k = 0; k < 6; ++k) {   // real parts only: (re.hi, re.lo) of each float4
      const float2* base = reinterpret_cast<const float2*>(EB + (size_t)k * g.G);
      const bool zc = (k % 3) == 2;
      const float2 v0 = base[2 * gn.off[0]], v1 = base[2 * gn.off[1]], v2 = base[2 * gn.off[2]],
                   v3 = base[2 * gn.off[3]];
      acc[k].s = 0.f;
      acc[k].c = 0.f;
      dot2_add(acc[k], zc ? w[0] : f0, v0.x, v0.y);
      dot2_add(acc[k], w[1], v1.x, v1.y);
      dot2_add(acc[k], zc ? w[2] : f2, v2.x, v2.y);
      dot2_add(acc[k], w[3], v3.x, v3.y);
    }
  }
  const dw c1 = dw_from_double(c), s1 = dw_from_double(s);
  dw cm = c1, sm = s1;   // cos(m theta), sin(m theta)
  for (int m = 1; m < g.Nm; ++m) {
    const dw c2 = dw_twice(cm), s2 = dw_twice(sm);
    dw A[4], S[4];
#pragma unroll
    for (int n = 0; n < 4; ++n) {
      A[n] = w[n] * c2;
      S[n] = w[n] * s2;
    }
    // fold signs of the inner nodes: z components (-1)^m, r and theta (-1)^{m+1}
    const bool negZ = gn.ghost && (m & 1), negV = gn.ghost && !(m & 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
      const float4* base = EB + (size_t)k * g.G + (size_t)m * RZ;
      const bool neg = (k % 3) == 2 ? negZ : negV;
      const float4 v0 = base[gn.off[0]], v1 = base[gn.off[1]], v2 = base[gn.off[2]], v3 = base[gn.off[3]];
      dot2_add(acc[k], neg_if(A[0], neg), v0.x, v0.y);
      dot2_add(acc[k], neg_if(S[0], neg), v0.z, v0.w);
      dot2_add(acc[k], A[1], v1.x, v1.y);
      dot2_add(acc[k], S[1], v1.z, v1.w);
      dot2_add(acc[k], neg_if(A[2], neg), v2.x, v2.y);
      dot2_add(acc[k], neg_if(S[2], neg), v2.z, v2.w);
      dot2_add(acc[k], A[3], v3.x, v3.y);
      dot2_add(acc[k], S[3], v3.z, v3.w);
    }
    const dw nc = cm * c1 - sm * s1, ns = sm * c1 + cm * s1;   // times e^{i theta}
    cm = nc;
    sm = ns;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) F[k] = dw_widen(acc[k].s) + dw_widen(acc[k].c);   // one rounding
}

// ------------------------------------------------------------------ a1: keys and sort
// Inactive particles (w = 0, moving window) take keys past the cells, Nz*Nr + ((i / 32) mod
// kTailBins): the sort gathers them at the end of the arrays, where whole chunks of them
// cost the band kernels nothing.  The 32 particles of one aligned group share a sub-bin, so
// each warp counts and places its inactive particles with one atomic (and the atomics of
// many warps spread over kTailBins addresses).
constexpr int kTailBins = 64;

__device__ __forceinline__ int tail_key(int ncell, int64_t i) { return ncell + (int)((i >> 5) & (kTailBins - 1)); }

// Warp-aggregated count of the inactive lanes of this iteration (all share one sub-bin).
__device__ __forceinline__ void count_inactive(int32_t* count, int key, bool inactive) {
  const unsigned am = __activemask();
  const unsigned m = __ballot_sync(am, inactive);
  if (inactive && (threadIdx.x & 31) == __ffs(m) - 1) atomicAdd(count + key, __popc(m));
}

// WIN (moving window on): inactive particles take the tail keys.
template <bool WIN>
__global__ void k_keys(const Parts p, int64_t np, GridGeom g, int32_t* keys, int32_t* count,
                       int32_t* err) {
  const int ncell = g.Nz * g.Nr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (WIN) {
      const bool inactive = p.w[i] == 0.0;
      count_inactive(count, tail_key(ncell, i), inactive);
      if (inactive) {
        keys[i] = tail_key(ncell, i);
        continue;
      }
    }
    double x = p.x[i], y = p.y[i], z = p.z[i];
    double r = sqrt(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)));
    double fz = floor(div_rn(z, g.dz, g.inv_dz)), fr = floor(div_rn(r, g.dr, g.inv_dr));
    if (!(fz == fz) || !(fr == fr) || isinf(fz) || isinf(fr)) {
      atomicOr(err, kErrNumeric);
      fz = 0.0; fr = 0.0;
    }
    int iz = (int)fmin(fmax(fz, 0.0), (double)(g.Nz - 1));
    int ir = (int)fmin(fmax(fr, 0.0), (double)(g.Nr - 1));
    int key = iz * g.Nr + ir;
    keys[i] = key;
    atomicAdd(count + key, 1);
  }
}

// exclusive scan of count[0..n) into start[0..n], 4096 elements per block
constexpr int kScanThreads = 1024, kScanPer = 4, kScanBlock = kScanThreads * kScanPer;

__device__ int32_t block_exclusive_scan(int32_t v, int32_t* total) {
  __shared__ int32_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int32_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int32_t w = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
    for (int o = 1; o < 32; o <<= 1) {
      int32_t y = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += y;
    }
    warp_sums[lane] = w;
  }
  __syncthreads();
  int32_t excl = x - v + (warp > 0 ? warp_sums[warp - 1] : 0);
  if (total) *total = warp_sums[(blockDim.x >> 5) - 1];
  __syncthreads();
  return excl;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_local(const int32_t* count, int32_t* start,
                                                              int32_t* blk, int n) {
  const int base = blockIdx.x * kScanBlock + threadIdx.x * kScanPer;
  int32_t v[kScanPer], sum = 0;
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = (base + q < n) ? count[base + q] : 0;
    sum += v[q];
  }
  int32_t tot;
  int32_t ex = block_exclusive_scan(sum, &tot);
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < n) start[base + q] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0) blk[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_blocks(int32_t* blk, int nblk, int32_t* start,
                                                               int n) {
  // one block: exclusive scan of up to 4096 block totals
  const int base = threadIdx.x * kScanPer;
  int32_t v[kScanPer], sum = 0;
  for (int q = 0; q < kScanPer; ++q) {
    v[q] = (base + q < nblk) ? blk[base + q] : 0;
    sum += v[q];
  }
  int32_t tot;
  int32_t ex = block_exclusive_scan(sum, &tot);
  for (int q = 0; q < kScanPer; ++q) {
    if (base + q < nblk) blk[base + q] = ex;
    ex += v[q];
  }
  if (threadIdx.x == 0) start[n] = tot;
}

__global__ void k_scan_add(int32_t* start, const int32_t* blk, int n, int32_t* cursor) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int32_t v = start[i] + blk[i / kScanBlock];
    start[i] = v;
    cursor[i] = v;
  }
}

// Counting-sort scatter; the inactive lanes of a warp iteration (one sub-bin, see tail_key)
// take their places with one atomic.
template <bool WIN>
__global__ void k_scatter(const int32_t* keys, int64_t np, int32_t* cursor, int32_t* tmp, int32_t ncell) {
  const int lane = threadIdx.x & 31;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t key = keys[i];
    if (!WIN) {
      tmp[atomicAdd(cursor + key, 1)] = (int32_t)i;
      continue;
    }
    const bool t = key >= ncell;
    const unsigned am = __activemask();
    const unsigned m = __ballot_sync(am, t);
    int32_t pos;
    if (t) {
      const int leader = __ffs(m) - 1;
      int32_t b = 0;
      if (lane == leader) b = atomicAdd(cursor + key, __popc(m));
      b = __shfl_sync(m, b, leader);
      pos = b + __popc(m & ((1u << lane) - 1u));
    } else {
      pos = atomicAdd(cursor + key, 1);
    }
    tmp[pos] = (int32_t)i;
  }
}

// Within each cell, order the particle indices ascending (this makes the counting sort
// stable and deterministic).  Cells with <= 16 particles: insertion sort by one thread;
// cells up to kWarpCellMax are queued at the front of big_list for a warp each, larger
// ones at its back for a CTA each (big_count[0], big_count[1]; cell_sort.cuh).
constexpr int kSmallCell = 16;
__global__ void k_cell_sort_small(const int32_t* start, const int32_t* tmp, int32_t* perm, int ncell,
                                  int32_t* big_list, int32_t* big_count) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    const int s0 = start[c], n = start[c + 1] - s0;
    if (n == 0) continue;
    if (n > kSmallCell) {
      if (n <= kWarpCellMax) big_list[atomicAdd(big_count, 1)] = c;
      else big_list[ncell - 1 - atomicAdd(big_count + 1, 1)] = c;
      continue;
    }
    int32_t v[kSmallCell];
    for (int k = 0; k < n; ++k) {
      int32_t e = tmp[s0 + k];
      int q = k;
      while (q > 0 && v[q - 1] > e) { v[q] = v[q - 1]; --q; }
      v[q] = e;
    }
    for (int k = 0; k < n; ++k) perm[s0 + k] = v[k];
  }
}

// With tail = 1 the inactive sub-bins past the ncell cells are copied over as they are
// (nothing depends on the order of inactive particles).  The cells queued at the back of
// big_list are sorted by whole CTAs, which use the cell's range of tmp as their second
// buffer.
__global__ void __launch_bounds__(256) k_cell_sort_big(const int32_t* start, int32_t* tmp, int32_t* perm,
                                                       const int32_t* big_list, const int32_t* big_count,
                                                       int ncell, int tail) {
  __shared__ int32_t sm[kCellChunk];
  if (tail) {
    const int32_t b = start[ncell], e = start[ncell + kTailBins];
    for (int32_t i = b + blockIdx.x * blockDim.x + threadIdx.x; i < e; i += gridDim.x * blockDim.x) perm[i] = tmp[i];
  }
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nw = (gridDim.x * blockDim.x) >> 5;
  const int nmid = big_count[0], nhuge = big_count[1];
  for (int b = gw; b < nmid; b += nw) {
    const int c = big_list[b];
    const int s0 = start[c];
    warp_rank_cell(tmp + s0, perm + s0, start[c + 1] - s0);
  }
  for (int b = blockIdx.x; b < nhuge; b += gridDim.x) {
    const int c = big_list[ncell - 1 - b];
    const int s0 = start[c];
    cta_sort_cell(tmp + s0, perm + s0, tmp + s0, start[c + 1] - s0, sm);
  }
}

// dst[i] = src[perm[i]]; with a moving window (slot non-null) the array index of every
// inactive particle is recorded by id for the next injection.
template <bool WIN>
__global__ void k_permute(const Parts src, Parts dst, const int32_t* perm, int64_t np, int32_t* slot) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t k = perm[i];
    const double w = src.w[k];
    const int32_t id = src.id[k];
    dst.x[i] = src.x[k]; dst.y[i] = src.y[k]; dst.z[i] = src.z[k];
    dst.ux[i] = src.ux[k]; dst.uy[i] = src.uy[k]; dst.uz[i] = src.uz[k];
    dst.w[i] = w; dst.id[i] = id;
    if (WIN && w == 0.0) slot[id] = (int32_t)i;
  }
}

// ------------------------------------------------------------------ a4: deposit
struct DepArgs {
  double2* rho;   // [Nm][Nr][Nz] or null
  double2* J;     // [3][Nm][Nr][Nz] or null
  double q;
  int32_t id_lo, id_hi;
};

// x with its sign flipped when neg (integer operations: the float64 unit bounds these kernels).
__device__ __forceinline__ double flip_sign(double x, bool neg) {
  return __longlong_as_double(__double_as_longlong(x) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}

__device__ __forceinline__ void dep2(double2* p, double re, double im) {
  double* d = reinterpret_cast<double*>(p);
  atomicAdd(d, re);
  atomicAdd(d + 1, im);
}

// Deposit of one particle: rho (do_rho) and/or J (do_J) with weight e^{+i m theta} per mode,
// linear weights; the ghost node r = -dr/2 of the axis cell is node 0 seen across the axis
// (fold sign (-1)^m for rho and J_z, (-1)^{m+1} for J_r and J_theta) and node Nr is dropped.
// The mode-independent products are formed once per node: g = q w w_z w_r / V_j and g v_k;
// each mode multiplies them by its phase (mode 0: real, so its imaginary parts, which would
// receive zeros, are left alone).  Lanes visit the 4 nodes in an order rotated by the lane
// index, so that lanes of one cell (same nodes) add to different nodes in one instruction.
// deposit_at takes the particle's radius and azimuth (r, cos, sin) already formed.
__device__ void deposit_at(const GridGeom& g, const DepArgs& a, const double* invV, double r,
                           double c, double s, double z, double w, double vx, double vy, double vz,
                           bool do_rho, bool do_J) {
  const Stencil st = stencil(g, z, r);
  const size_t RZ = (size_t)g.Nr * g.Nz;
  const int rot = threadIdx.x & 3;
  const bool ghost = st.j0 < 0;
  const double qw = a.q * w;
  double rad[2];   // q w w_r / V_j of the radial nodes j0, j0 + 1 (0 for the dropped node Nr)
  int jn[2];       // their grid rows (the ghost node j = -1 is row 0)
#pragma unroll
  for (int dj = 0; dj < 2; ++dj) {
    const int j = st.j0 + dj;
    const bool keep = j < g.Nr;
    jn[dj] = (j < 0 || !keep) ? 0 : j;
    rad[dj] = keep ? (dj ? st.wr1 : st.wr0) * (invV[jn[dj]] * qw) : 0.0;
  }
  const double vr = c * vx + s * vy, vt = c * vy - s * vx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int node = (q + rot) & 3, dz = node >> 1, dj = node & 1;
    const double gq = (dz ? st.wz1 : st.wz0) * (dj ? rad[1] : rad[0]);
    if (gq == 0.0) continue;
    const size_t o = (size_t)(dj ? jn[1] : jn[0]) * g.Nz + (dz ? st.i1 : st.i0);
    const bool fold = ghost && dj == 0;   // the ghost node: fold signs apply
    double gr = 0.0, gt = 0.0, gz = 0.0;
    if (do_J) {
      gr = gq * vr;
      gt = gq * vt;
      gz = gq * vz;
    }
    // mode 0: fold +1 for rho and J_z, -1 for J_r and J_theta
    if (do_rho) atomicAdd(reinterpret_cast<double*>(a.rho + o), gq);
    if (do_J) {
      atomicAdd(reinterpret_cast<double*>(a.J + o), flip_sign(gr, fold));
      atomicAdd(reinterpret_cast<double*>(a.J + g.G + o), flip_sign(gt, fold));
      atomicAdd(reinterpret_cast<double*>(a.J + 2 * g.G + o), gz);
    }
    double pr = c, pi = s;   // e^{+i m theta}
    for (int m = 1; m < g.Nm; ++m) {
      const bool negS = fold && (m & 1), negV = fold && !(m & 1);
      const size_t om = (size_t)m * RZ + o;
      if (do_rho) {
        const double v = flip_sign(gq, negS);
        dep2(a.rho + om, v * pr, v * pi);
      }
      if (do_J) {
        const double jr = flip_sign(gr, negV), jt = flip_sign(gt, negV), jz = flip_sign(gz, negS);
        dep2(a.J + om, jr * pr, jr * pi);
        dep2(a.J + g.G + om, jt * pr, jt * pi);
        dep2(a.J + 2 * g.G + om, jz * pr, jz * pi);
      }
      if (m + 1 < g.Nm) {
        const double nr = pr * c - pi * s, ni = pr * s + pi * c;
        pr = nr;
        pi = ni;
      }
    }
  }
}

__device__ __forceinline__ void deposit_one(const GridGeom& g, const DepArgs& a, const double* invV,
                                            double x, double y, double z, double w, double vx,
                                            double vy, double vz, bool do_rho, bool do_J) {
  double r, c, s;
  polar(x, y, r, c, s);
  deposit_at(g, a, invV, r, c, s, z, w, vx, vy, vz, do_rho, do_J);
}

__global__ void k_deposit(const Parts p, int64_t np, GridGeom g, DepArgs a, const double* invV,
                          int32_t* err) {
  const bool do_rho = a.rho != nullptr, do_J = a.J != nullptr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t id = p.id[i];
    if (id < a.id_lo || id >= a.id_hi) continue;
    double vx = 0.0, vy = 0.0, vz = 0.0;
    if (do_J) {
      const double ux = p.ux[i], uy = p.uy[i], uz = p.uz[i];
      const double ig = rsqrt(1.0 + (ux * ux + uy * uy + uz * uz) * kInvC2);
      vx = ux * ig; vy = uy * ig; vz = uz * ig;
    }
    const double wt = p.w[i];
    if (wt == 0.0) continue;   // inactive particles add nothing
    const double x = p.x[i], y = p.y[i], z = p.z[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) { atomicOr(err, kErrNumeric); continue; }
    deposit_one(g, a, invV, x, y, z, wt, vx, vy, vz, do_rho, do_J);
  }
}

__global__ void k_inv_volume(double* invV, int Nr, double dr, double dz) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < Nr) invV[j] = 1.0 / (2.0 * kPi * ((j + 0.5) * dr) * dr * dz);
}

// ------------------------------------------------------------------ a2 + a3 (+ a4 J)
// Moving window: record a particle that became inactive (flag and slot by id, count per block
// of 1024 ids).  The records persist: the permute keeps the slots of inactive particles
// current and the injection clears the records it uses.
__device__ __forceinline__ void win_mark(const WinArgs& wa, int32_t id, int64_t i) {
  wa.flag[id] = 1;
  wa.slot[id] = (int32_t)i;
  atomicAdd(wa.bcnt + (id >> 10), 1);
}

// WIN: moving window on (removal behind the back edge); the plain instance has none of it.
// DWG: gather from the double-word copy of E, B (gather_dw) instead of the float64 grids.
template <bool WIN, bool DWG>
__global__ void __launch_bounds__(256, 2) k_gather_push(Parts p, int64_t np, GridGeom g, const double2* __restrict__ E,
                              const double2* __restrict__ B, const float4* __restrict__ EBdw, double k,
                              double dt, DepArgs dep, const double* invV, int fuse, int32_t* err,
                              WinArgs wa) {
  const size_t RZ = (size_t)g.Nr * g.Nz;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double w = p.w[i];
    if (w == 0.0) continue;   // inactive (moving window): neither pushed nor moved
    double x = p.x[i], y = p.y[i], z = p.z[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(z)) { atomicOr(err, kErrNumeric); continue; }
    const double z_old = z;
    double ux = p.ux[i], uy = p.uy[i], uz = p.uz[i];
    double r, c, s;
    polar(x, y, r, c, s);
    const Stencil st = stencil(g, z, r);
    // F = Re sum_m mult_m e^{-i m theta} sum_n w_n F_m(node n), mult_0 = 1, mult_m = 2; per
    // mode the node weights are multiplied by mult e^{-i m theta} once for the 6 components,
    // and the ghost nodes (n = 0, 2) are summed apart so that the fold is one sign flip.
    const GatherNodes gn = gather_nodes(g, st);
    double F[6];   // E_r, E_t, E_z, B_r, B_t, B_z
    if constexpr (DWG) {
      gather_dw(g, gn, c, s, EBdw, F);
    } else {
#pragma unroll
    for (int k = 0; k < 6; ++k) {   // mode 0: real phase, fold +1 for E_z, B_z and -1 for r, theta
      const double2* base = (k < 3 ? E : B) + (size_t)(k % 3) * g.G;
      const double in = gn.w[0] * base[gn.off[0]].x + gn.w[2] * base[gn.off[2]].x;
      const double out = gn.w[1] * base[gn.off[1]].x + gn.w[3] * base[gn.off[3]].x;
      F[k] = out + flip_sign(in, gn.ghost && (k % 3) != 2);
    }
    double phr = c, phi = -s;   // e^{-i m theta}, m = 1
    for (int m = 1; m < g.Nm; ++m) {
      double a[4], b[4];
#pragma unroll
      for (int n = 0; n < 4; ++n) {
        a[n] = 2.0 * gn.w[n] * phr;
        b[n] = 2.0 * gn.w[n] * phi;
      }
      const bool negS = gn.ghost && (m & 1), negV = gn.ghost && !(m & 1);
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        const double2* base = (k < 3 ? E : B) + (size_t)(k % 3) * g.G + (size_t)m * RZ;
        const double2 v0 = base[gn.off[0]], v1 = base[gn.off[1]], v2 = base[gn.off[2]], v3 = base[gn.off[3]];
        const double in = a[0] * v0.x - b[0] * v0.y + a[2] * v2.x - b[2] * v2.y;
        const double out = a[1] * v1.x - b[1] * v1.y + a[3] * v3.x - b[3] * v3.y;
        F[k] += out + flip_sign(in, (k % 3) == 2 ? negS : negV);
      }
      const double nr = phr * c + phi * s, ni = phi * c - phr * s;   // times e^{-i theta}
      phr = nr; phi = ni;
    }
    }
    const double Ex = F[0] * c - F[1] * s, Ey = F[0] * s + F[1] * c, Ez = F[2];
    const double Bx = F[3] * c - F[4] * s, By = F[3] * s + F[4] * c, Bz = F[5];
    // Boris with k = q dt / (2 m) (from the host); 1/gamma^- once for the three t
    const double umx = ux + k * Ex, umy = uy + k * Ey, umz = uz + k * Ez;
    const double igm = rsqrt(1.0 + (umx * umx + umy * umy + umz * umz) * kInvC2);
    const double kb = k * igm;
    const double tx = kb * Bx, ty = kb * By, tz = kb * Bz;
    const double upx = umx + (umy * tz - umz * ty);
    const double upy = umy + (umz * tx - umx * tz);
    const double upz = umz + (umx * ty - umy * tx);
    const double f = 2.0 / (1.0 + tx * tx + ty * ty + tz * tz);
    const double sx = f * tx, sy = f * ty, sz = f * tz;
    ux = umx + (upy * sz - upz * sy) + k * Ex;
    uy = umy + (upz * sx - upx * sz) + k * Ey;
    uz = umz + (upx * sy - upy * sx) + k * Ez;
    const double ig = rsqrt(1.0 + (ux * ux + uy * uy + uz * uz) * kInvC2);
    const double vx = ux * ig, vy = uy * ig, vz = uz * ig;
    const double hdt = 0.5 * dt;
    x = __dadd_rn(x, __dmul_rn(hdt, vx));   // no FMA: one ulp of z is ~L/dz ulps of a weight
    y = __dadd_rn(y, __dmul_rn(hdt, vy));
    z = __dadd_rn(z, __dmul_rn(hdt, vz));
    if (z >= g.L) z -= g.L;
    if (z < 0.0) z += g.L;
    if (fuse) deposit_one(g, dep, invV, x, y, z, w, vx, vy, vz, false, true);
    x = __dadd_rn(x, __dmul_rn(hdt, vx));   // no FMA: one ulp of z is ~L/dz ulps of a weight
    y = __dadd_rn(y, __dmul_rn(hdt, vy));
    z = __dadd_rn(z, __dmul_rn(hdt, vz));
    if (z >= g.L) z -= g.L;
    if (z < 0.0) z += g.L;
    // one polar decomposition at x^{n+1} serves the wall and the rho deposit
    double r1, c1, s1;
    polar(x, y, r1, c1, s1);
    if (r1 >= g.R) {   // specular reflection (rare: the particle crossed the wall)
      const double fr = (2.0 * g.R - r1) / r1;
      const double ur = ux * c1 + uy * s1;
      ux = ux - 2.0 * ur * c1;
      uy = uy - 2.0 * ur * s1;
      x *= fr;
      y *= fr;
      polar(x, y, r1, c1, s1);
    }
    // rho^{n+1} at x^{n+1} (without the moving window; with it the deposit stage runs after
    // the injection)
    if (!WIN && dep.rho) deposit_at(g, dep, invV, r1, c1, s1, z, w, 0.0, 0.0, 0.0, true, false);
    if (WIN) {
      // window coordinate after the step: ((z^n - back) mod L) + 2 half moves - s dz
      double zo = z_old - wa.back_z;
      if (zo < 0.0) zo += g.L;
      const double d = __dmul_rn(hdt, vz);
      const double zn = __dsub_rn(__dadd_rn(__dadd_rn(zo, d), d), wa.shift ? g.dz : 0.0);
      if (zn < 0.0) {   // left through the back edge: inactive from now on
        p.w[i] = 0.0;
        ux = 0.0; uy = 0.0; uz = 0.0;
        win_mark(wa, p.id[i], i);
      }
    }
    p.x[i] = x; p.y[i] = y; p.z[i] = z;
    p.ux[i] = ux; p.uy[i] = uy; p.uz[i] = uz;
  }
}

// ------------------------------------------------------------------ a10: diagnostics
constexpr int kDiagThreads = 256;
constexpr int kMaxSlices = 1 << 16;

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ------------------------------------------------------------------ mixed form: FP32 particles
// Positions are kept relative to their cell: z = (iz + fz) dz with iz an int32 cell and
// x = (ix + fx) dr, y = (iy + fy) dr with (ix, iy) two int16 packed in one int32, and the
// fractions fz, fx, fy in [0, 1): a float fraction resolves 2^-24 of a cell anywhere in the
// box, where a float coordinate in metres loses precision away from the origin.  Momenta
// are u/c as float pairs hi + lo (|lo| <= ulp(hi)/2, 48 significant bits): a per-step kick
// of a gamma = 2000 beam is about one ulp of a float u/c, so a single float would round the
// beam's energy changes away.  w is float.
struct PartsF {
  int32_t* iz; float* fz; int32_t* ixy; float* fx; float* fy;
  float* ux; float* uy; float* uz; float* uxl; float* uyl; float* uzl; float* w; int32_t* id;
};

PartsF partsf_of(Sim* s, int which) {
  PartsF p;
  p.iz = s->at<int32_t>(s->lay.pf[which][kPfIz]);
  p.fz = s->at<float>(s->lay.pf[which][kPfFz]);
  p.ixy = s->at<int32_t>(s->lay.pf[which][kPfIxy]);
  p.fx = s->at<float>(s->lay.pf[which][kPfFx]);
  p.fy = s->at<float>(s->lay.pf[which][kPfFy]);
  p.ux = s->at<float>(s->lay.pf[which][kPfUx]);
  p.uy = s->at<float>(s->lay.pf[which][kPfUy]);
  p.uz = s->at<float>(s->lay.pf[which][kPfUz]);
  p.uxl = s->at<float>(s->lay.pf[which][kPfUxLo]);
  p.uyl = s->at<float>(s->lay.pf[which][kPfUyLo]);
  p.uzl = s->at<float>(s->lay.pf[which][kPfUzLo]);
  p.w = s->at<float>(s->lay.pf[which][kPfW]);
  p.id = s->at<int32_t>(s->lay.pf[which][kPfId]);
  return p;
}

__host__ __device__ __forceinline__ int32_t pack_cells(int ix, int iy) {
  return (int32_t)(((uint32_t)ix & 0xffffu) | ((uint32_t)iy << 16));
}
__device__ __forceinline__ int cell_x(int32_t v) { return (int)(int16_t)(v & 0xffff); }
__device__ __forceinline__ int cell_y(int32_t v) { return v >> 16; }

// (hi, lo) += b for a float pair (two-sum, then renormalisation)
__device__ __forceinline__ void ff_add(float& h, float& l, float b) {
  const float s = h + b;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (b - bb);
  const float t = l + e;
  h = s + t;
  l = t - (h - s);
}

// Advance a cell-relative coordinate (cell, fraction in [0, 1)) by d cells.
__device__ __forceinline__ void advance_cell(int& cell, float& f, float d) {
  f += d;
  const float k = floorf(f);
  f -= k;
  if (f >= 1.f) { f -= 1.f; cell += 1; }   // rounding of f - k up to 1
  cell += (int)k;
}

// x / dr and y / dr of particle i
__device__ __forceinline__ void pos_cells(const PartsF& p, int64_t i, float& x, float& y) {
  const int32_t c = p.ixy[i];
  x = (float)cell_x(c) + p.fx[i];
  y = (float)cell_y(c) + p.fy[i];
}

// Positions are handled in cell units (x / dr, y / dr) on the device.
struct GeomF {
  int Nz, Nr, Nm;
  size_t G;
};

GeomF geomf_of(const Sim* s) {
  const pic_config& c = s->cfg;
  GeomF g{c.Nz, c.Nr, c.Nm, s->grid_elems()};
  return g;
}

// ------------------------------------------------------------------ mixed form: gather layout
// E and B of every mode at one node, contiguous: ebn[(i Nr + j) NV + c Nm + m] with
// NV = 6 Nm and c = E_r, E_theta, E_z, B_r, B_theta, B_z.  A particle's 4 nodes are then
// two runs (z rows i0, i1) of two adjacent nodes, each node one 16-byte-aligned run of NV
// complex values read with vector loads.  Built from the [c][m][r][z] planes by
// k_nodes_rz through shared memory, in tiles of 32 z x tr r nodes and all NV planes.
// The same launch clears the current grids for the push's deposit (n_zero values from
// zero2) and starts the charge grid from the ion background (n_copy values, csrc2 to
// cdst2), spread over all its threads, so that no separate memset and copy run.
__global__ void __launch_bounds__(256) k_nodes_rz(const float2* __restrict__ src, float2* __restrict__ dst, int Nr,
                                                  int Nz, int NV, int tr, float2* __restrict__ zero2, int n_zero,
                                                  float2* __restrict__ cdst2, const float2* __restrict__ csrc2,
                                                  int n_copy) {
  extern __shared__ float2 node_tile[];   // [32][tr NV + 1]: odd pitch, conflict-free columns
  {
    const int nthr = gridDim.x * gridDim.y * blockDim.x;
    const int t0 = (blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + threadIdx.x;
    for (int i = t0; i < n_zero; i += nthr) zero2[i] = make_float2(0.f, 0.f);
    for (int i = t0; i < n_copy; i += nthr) cdst2[i] = csrc2[i];
  }
  const int pitch = tr * NV + 1;
  const int z0 = blockIdx.x * 32, r0 = blockIdx.y * tr;
  const int nr = min(tr, Nr - r0), nz = min(32, Nz - z0);
  const int RZ = Nr * Nz;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int q = ty; q < NV * tr; q += 8) {
    const int v = q / tr, rr = q - v * tr;
    if (rr < nr && tx < nz) node_tile[tx * pitch + rr * NV + v] = src[v * RZ + (r0 + rr) * Nz + z0 + tx];
  }
  __syncthreads();
  const int run = nr * NV;   // contiguous output values of one z row
  for (int e = threadIdx.x; e < nz * run; e += 256) {
    const int zz = e / run, k = e - zz * run;
    dst[((z0 + zz) * Nr + r0) * NV + k] = node_tile[zz * pitch + k];
  }
}

// Radial nodes of a particle at r (in cells; node j sits at r = j + 1/2) as a pair of
// adjacent nodes jb, jb + 1 with weights.  Node jb has one weight per fold class: in the
// axis cell (r < 1/2) the ghost node r = -1/2 is node 0 seen across the axis, so node 0
// carries wr1 + wr0 (class P: scalars and z components of even modes, r and theta
// components of odd modes) or wr1 - wr0 (class M: the others), and node 1 nothing.  In
// the last cell node Nr is dropped (jb = Nr - 2 carries nothing).  Needs Nr >= 2.
struct RadW {
  int jb;
  float aP, aM, b;
};

__device__ __forceinline__ RadW radial_nodes(float r, int Nr) {
  const float v = r - 0.5f;
  const float fj = floorf(v);
  const float t = v - fj;   // weight of node j0 + 1
  const int j0 = (int)fj;   // >= -1 for r >= 0
  RadW w;
  if (j0 < 0) {
    w.jb = 0; w.aP = 1.f; w.aM = 2.f * t - 1.f; w.b = 0.f;
  } else if (j0 >= Nr - 1) {
    w.jb = Nr - 2; w.aP = 0.f; w.aM = 0.f; w.b = j0 == Nr - 1 ? 1.f - t : 0.f;
  } else {
    w.jb = j0; w.aP = 1.f - t; w.aM = w.aP; w.b = t;
  }
  return w;
}

// Fold class of component type zlike (scalars, z components) in mode m: P when the ghost
// node's sign is +1 ((-1)^m for zlike, -(-1)^m for r and theta components).
__host__ __device__ constexpr bool class_p(bool zlike, int m) { return zlike == ((m & 1) == 0); }

// r, cos(theta), sin(theta) of (x, y) in cells (theta = 0 on the axis).
__device__ __forceinline__ void polar_rcp(float x, float y, float& r, float& c, float& s) {
  const float r2 = __fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y));
  if (r2 > 0.f) {
    const float ir = rsqrtf(r2);
    r = r2 * ir; c = x * ir; s = y * ir;
  } else {
    r = 0.f; c = 1.f; s = 0.f;
  }
}

// Fields at a particle: F = (E_r, E_theta, E_z, B_r, B_theta, B_z) of
// Re[F_0 + 2 sum_{m>=1} F_m e^{-i m theta}] interpolated linearly from the 4 nodes.
template <int NM>
__device__ __forceinline__ void gather_nodes(const float2* __restrict__ ebn, int Nr, int i0, int i1, float wz0,
                                             float wz1, const RadW& rw, float c, float s, float F[6]) {
  constexpr int NV = 6 * NM;
  float pr[NM], pi[NM];   // e^{-i m theta}, then times the mode multiplicity (2 for m >= 1)
  pr[0] = 1.f; pi[0] = 0.f;
#pragma unroll
  for (int m = 1; m < NM; ++m) {
    pr[m] = pr[m - 1] * c + pi[m - 1] * s;
    pi[m] = pi[m - 1] * c - pr[m - 1] * s;
  }
#pragma unroll
  for (int m = 1; m < NM; ++m) { pr[m] *= 2.f; pi[m] *= 2.f; }
#pragma unroll
  for (int k = 0; k < 6; ++k) F[k] = 0.f;
#pragma unroll
  for (int row = 0; row < 2; ++row) {
    const float wz = row ? wz1 : wz0;
    const float4* nd = reinterpret_cast<const float4*>(ebn + ((row ? i1 : i0) * Nr + rw.jb) * NV);
#pragma unroll
    for (int node = 0; node < 2; ++node) {
      const float wP = wz * (node ? rw.b : rw.aP), wM = wz * (node ? rw.b : rw.aM);
#pragma unroll
      for (int q = 0; q < NV / 2; ++q) {
        const float4 d = __ldg(nd + node * (NV / 2) + q);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int v = 2 * q + h, comp = v / NM, m = v - comp * NM;
          const float w = class_p(comp % 3 == 2, m) ? wP : wM;
          const float re = h ? d.z : d.x, im = h ? d.w : d.y;
          F[comp] = fmaf(w * pr[m], re, F[comp]);
          F[comp] = fmaf(-w * pi[m], im, F[comp]);
        }
      }
    }
  }
}

struct DepArgsF {
  float2* rho;   // [Nm][Nr][Nz] or null
  float2* J;     // [3][Nm][Nr][Nz] (J_r, J_theta, J_z) or null
  float q;
  int32_t id_lo, id_hi;
};

// Shared-memory band of a CTA: TZ z rows (a power of two) from row iz_lo and JW r nodes
// from node j_lo, node-major.  Node (row, jj) starts at word row RS + jj NWP; it holds NC
// components (rho first when the band carries it, then J_r, J_theta, J_z), each with, per
// mode, two int32 words (hi, lo) of the real part and, for m >= 1, two of the imaginary
// part (mode 0 has a real phase): CW = 4 Nm - 2 words per component.  NWP = NC CW + 1 is
// odd, so that consecutive nodes start in different banks, and the row stride RS is
// padded to RS mod 32 = 8, so that the 4 rows read together by the flush do too.
//
// Values are 48-bit fixed point: a contribution x (charge times weights, before the 1/V_j
// factor) becomes y = x 2^S rounded to an integer, y = 2^16 hi + lo with |lo| <= 2^15,
// and hi and lo are added with integer shared-memory atomics (native, where float ones
// are compare-and-swap loops, and independent of the order of the adds).  S is chosen per
// CTA so that |y| <= 2^(46 - log2 chunk) for every contribution of its chunk; an entry
// takes at most one add per particle, so |sum y| <= 2^46, |sum hi| < 2^31 and
// |sum lo| <= 2^(15 + log2 chunk).  rho has its own scale (scale0).
struct BandF {
  int32_t* tile;   // null: no band, every deposit goes to the global grids
  int iz_lo, TZ, lgTZ, j_lo, JW, RS;
  float scale, scale0;
};

__host__ __device__ constexpr int band_node_words(int nm, int nc) { return nc * (4 * nm - 2) + 1; }
__host__ __device__ constexpr int mode_word(int m) { return m == 0 ? 0 : 4 * m - 2; }

// Launch-wide band parameters: chunk of particles per CTA, at most tz rows (a power of two,
// 0: no band) and jw_max r nodes; jmargin = r nodes a particle can move before it deposits.
struct BandArgs {
  int64_t chunk;
  int tz, jw_max, jmargin;
  int lg_chunk;   // log2 chunk: sets the fixed-point headroom
};

// Per-chunk statistics gathered before a band is laid out.
struct ChunkStats {
  uint32_t wmax_bits;   // largest |w| (non-negative float bits)
  int jmin, jmax;       // range of the particles' lower radial stencil node floor(r/dr - 1/2)
};

constexpr float kFxHi = 824633720832.f;   // 1.5 2^39: adding it rounds |y| < 2^38 to a multiple of 2^16
constexpr float kFxLo = 12582912.f;       // 1.5 2^23: adding it rounds |d| < 2^22 to an integer

// Adds a ws, rounded to 48-bit fixed point, to the word pair p[0] (hi), p[1] (lo).  The
// split uses the magic-number sums above (float adds and integer subtractions of the bit
// patterns): t - kFxHi = round(a ws / 2^16) 2^16 exactly, and d = a ws - (t - kFxHi) is
// exact within one rounding and below 2^15 + 1 in magnitude.
__device__ __forceinline__ void fx_add(int32_t* p, float a, float ws) {
  const float t = fmaf(a, ws, kFxHi);
  const float d = fmaf(a, ws, -(t - kFxHi));
  atomicAdd(p, __float_as_int(t) - __float_as_int(kFxHi));
  atomicAdd(p + 1, __float_as_int(d + kFxLo) - __float_as_int(kFxLo));
}

// 2^16 hi + lo as the correctly rounded float, with 32-bit integer operations only: the
// carry of lo moves into hi, then the sum is (h >> 8) 2^24 + ((h & 255) 2^16 + (lo & 65535)),
// two terms that floats hold exactly, added by one fused multiply-add.
__device__ __forceinline__ float fx_value(int32_t hi, int32_t lo) {
  const int32_t h = hi + (lo >> 16);
  const int32_t l = lo & 0xffff;
  return fmaf((float)(h >> 8), 16777216.f, (float)(((h & 0xff) << 16) | l));
}

// Largest |w| and radial stencil range over particles [b0, b1) (all threads of the CTA;
// non-finite weights raise the numeric error bit and count as 0).
__device__ __forceinline__ ChunkStats chunk_stats(const PartsF& p, const GeomF& g, int64_t b0, int64_t b1,
                                                  ChunkStats* slot, int32_t* err) {
  if (threadIdx.x == 0) *slot = ChunkStats{0u, g.Nr, -1};
  __syncthreads();
  float mx = 0.f;
  int jmin = g.Nr, jmax = -1;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    float a = fabsf(p.w[i]);
    if (!(a <= 3.0e38f)) { atomicOr(err, kErrNumeric); a = 0.f; }
    mx = fmaxf(mx, a);
    float x, y;
    pos_cells(p, i, x, y);
    const float v = sqrtf(x * x + y * y) - 0.5f;
    const int j = (int)fminf(fmaxf(floorf(v), -1.f), (float)g.Nr);   // NaN -> -1 after fmaxf
    jmin = min(jmin, j);
    jmax = max(jmax, j);
  }
  // non-negative floats order like their bit patterns
  const uint32_t m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
  jmin = __reduce_min_sync(0xffffffffu, jmin);
  jmax = __reduce_max_sync(0xffffffffu, jmax);
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&slot->wmax_bits, m);
    atomicMin(&slot->jmin, jmin);
    atomicMax(&slot->jmax, jmax);
  }
  __syncthreads();
  return *slot;
}

// Band of a chunk of cell-sorted particles whose first and last cells are iz_first, iz_last:
// rows from iz_first - 1 to iz_last + 2 (moves of up to half a cell per half step, and the
// +1 node), at most tz_max rows; r nodes from the chunk's lowest stencil node - jmargin to
// its highest + 1 + jmargin (at least 2, at most jw_max); particles whose nodes are not all
// inside deposit to the global grids.  bound (bound0) is an upper bound of |x| over the
// chunk's J (rho) contributions.
__device__ __forceinline__ BandF make_band(int32_t* smem, int iz_first, int iz_last, const GeomF& g, int tz_max,
                                           int nwp, const ChunkStats& cs, int jw_max, int jmargin, int lg_chunk,
                                           float bound, float bound0) {
  const int j_lo = min(max(0, cs.jmin - jmargin), g.Nr - 2);
  const int j_hi = min(g.Nr - 1, max(cs.jmax + 1 + jmargin, j_lo + 1));
  const int JW = max(2, min(jw_max, j_hi - j_lo + 1));
  if (iz_first < 0 || iz_first >= g.Nz) iz_first = 0;
  if (iz_last < 0 || iz_last >= g.Nz) iz_last = iz_first;
  int span = iz_last - iz_first;
  if (span < 0) span += g.Nz;
  int lg = 2;   // rows: the smallest power of two >= span + 4, at most tz_max (a power of two)
  while ((1 << lg) < span + 4 && (2 << lg) <= tz_max) ++lg;
  int e = 0;
  frexpf(bound, &e);   // bound <= 2^e
  const int S = min(max(46 - lg_chunk - e, -126), 126);
  frexpf(bound0, &e);
  const int S0 = min(max(46 - lg_chunk - e, -126), 126);
  int RS = JW * nwp;
  RS += (40 - RS % 32) % 32;   // RS mod 32 = 8
  return BandF{smem, iz_first == 0 ? g.Nz - 1 : iz_first - 1, 1 << lg, lg, j_lo, JW, RS, ldexpf(1.f, S),
               ldexpf(1.f, S0)};
}

// Zero a band (all threads of the CTA).
__device__ __forceinline__ void band_zero(const BandF& bd) {
  if (!bd.tile) return;
  const int n = bd.TZ * bd.RS;
  for (int k = threadIdx.x; k < n; k += blockDim.x) bd.tile[k] = 0;
}

// Fixed-point adds of one node: rho (DO_RHO, component 0) and J (DO_J, components NC-3..NC-1).
// sP, sM: the node's weight in fold classes P and M; qr, qi: charge times e^{+i m theta};
// vel: (v_r, v_theta, v_z).
template <int NM, int NC, bool DO_RHO, bool DO_J>
__device__ __forceinline__ void band_node(int32_t* e, float sP, float sM, const BandF& bd, const float* qr,
                                          const float* qi, const float* vel) {
  constexpr int CW = 4 * NM - 2;
  if (DO_RHO) {
    const float wP = sP * bd.scale0, wM = sM * bd.scale0;
#pragma unroll
    for (int m = 0; m < NM; ++m) {
      const float ws = class_p(true, m) ? wP : wM;
      fx_add(e + mode_word(m), qr[m], ws);
      if (m) fx_add(e + mode_word(m) + 2, qi[m], ws);
    }
  }
  if (DO_J) {
    const float wP = sP * bd.scale, wM = sM * bd.scale;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      int32_t* ek = e + (NC - 3 + k) * CW;
#pragma unroll
      for (int m = 0; m < NM; ++m) {
        const float ws = class_p(k == 2, m) ? wP : wM;
        fx_add(ek + mode_word(m), vel[k] * qr[m], ws);
        if (m) fx_add(ek + mode_word(m) + 2, vel[k] * qi[m], ws);
      }
    }
  }
}

// One node's contributions straight into the global grids (float atomics, 1/V_j applied):
// the path of the nodes that lie outside a CTA's band.
template <int NM, bool DO_RHO, bool DO_J>
__device__ __forceinline__ void global_node(const GeomF& g, const DepArgsF& a, const float* invV, int i, int j,
                                            float sP, float sM, const float* qr, const float* qi, const float* vel) {
  const int RZ = g.Nr * g.Nz, G = (int)g.G;
  const float iv = invV[j];
  const int off = j * g.Nz + i;
#pragma unroll
  for (int m = 0; m < NM; ++m) {
    if (DO_RHO) {
      const float f = (class_p(true, m) ? sP : sM) * iv;
      atomicAdd(a.rho + m * RZ + off, make_float2(qr[m] * f, qi[m] * f));
    }
    if (DO_J) {
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        const float f = (class_p(k == 2, m) ? sP : sM) * iv * vel[k];
        atomicAdd(a.J + k * G + m * RZ + off, make_float2(qr[m] * f, qi[m] * f));
      }
    }
  }
}

// Deposit of one particle at (iz + fz, x, y) (cells) with weight w and velocity
// (vx, vy, vz) [m/s]: rho (DO_RHO) and/or J (DO_J) with weight e^{+i m theta} per mode
// (the projection onto the e^{-i m theta} modes), linear weights, the axis fold of the
// ghost node and node Nr dropped (radial_nodes).  Each node goes into the band when it lies
// inside, else straight into the global grids.  Lanes visit the 4 nodes in an order
// rotated by the lane index, so that lanes of one cell (which share their nodes) add to
// different nodes in the same instruction.
template <int NM, int NC, bool DO_RHO, bool DO_J>
__device__ __forceinline__ void deposit_nodes(const BandF& bd, const GeomF& g, const DepArgsF& a, const float* invV,
                                              int iz, float fz, float x, float y, float w, float vx, float vy,
                                              float vz) {
  constexpr int NWP = band_node_words(NM, NC);
  float r, c, s;
  polar_rcp(x, y, r, c, s);
  const RadW rw = radial_nodes(r, g.Nr);
  float qr[NM], qi[NM];
  qr[0] = a.q * w; qi[0] = 0.f;
#pragma unroll
  for (int m = 1; m < NM; ++m) {
    qr[m] = qr[m - 1] * c - qi[m - 1] * s;
    qi[m] = qr[m - 1] * s + qi[m - 1] * c;
  }
  const float vel[3] = {c * vx + s * vy, c * vy - s * vx, vz};
  int row0 = iz - bd.iz_lo;
  if (row0 < 0) row0 += g.Nz;
  const int jj = rw.jb - bd.j_lo;
  const int rot = threadIdx.x & 3;
#pragma unroll 1
  for (int q = 0; q < 4; ++q) {
    const int node = (q + rot) & 3, row = node >> 1, nb = node & 1;
    const float wz = row ? fz : 1.f - fz;
    const float sP = wz * (nb ? rw.b : rw.aP), sM = wz * (nb ? rw.b : rw.aM);
    if (sP == 0.f && sM == 0.f) continue;
    const int brow = row0 + row, bj = jj + nb;
    if (bd.tile && brow < bd.TZ && (unsigned)bj < (unsigned)bd.JW)
      band_node<NM, NC, DO_RHO, DO_J>(bd.tile + brow * bd.RS + bj * NWP, sP, sM, bd, qr, qi, vel);
    else
      global_node<NM, DO_RHO, DO_J>(g, a, invV, row ? (iz + 1 == g.Nz ? 0 : iz + 1) : iz, rw.jb + nb, sP, sM, qr,
                                    qi, vel);
  }
}

// Add a band's non-zero entries, times 2^-S / V_j, to the global grids (all threads of the
// CTA): rho (component 0 when RHO0) and J_r, J_theta, J_z (the next three, G apart in J).
// Consecutive threads take consecutive rows of one (node, component, mode), adjacent in
// global memory.
template <int NM, int NC, bool RHO0>
__device__ void band_flush(const BandF& bd, const GeomF& g, float2* rho, float2* J, const float* invV) {
  if (!bd.tile) return;
  constexpr int CW = 4 * NM - 2, NWP = band_node_words(NM, NC), NCM = NC * NM;
  const int RZ = g.Nr * g.Nz, G = (int)g.G;
  const float inv_s = 1.f / bd.scale, inv_s0 = 1.f / bd.scale0;   // powers of two: exact
  const int total = (bd.JW * NCM) << bd.lgTZ;
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int row = idx & (bd.TZ - 1);
    const int q = idx >> bd.lgTZ;
    const int jj = q / NCM;
    const int cm = q - jj * NCM;
    const int k = cm / NM, m = cm - k * NM;
    const int32_t* e = bd.tile + row * bd.RS + jj * NWP + k * CW + mode_word(m);
    const int32_t hr = e[0], lr = e[1];
    const int32_t hi = m ? e[2] : 0, li = m ? e[3] : 0;
    if ((hr | lr | hi | li) == 0) continue;
    const int j = bd.j_lo + jj;
    const float f = (RHO0 && k == 0 ? inv_s0 : inv_s) * invV[j];
    int i = bd.iz_lo + row;
    if (i >= g.Nz) i -= g.Nz;
    float2* grid = RHO0 && k == 0 ? rho : J + (k - (RHO0 ? 1 : 0)) * G;
    atomicAdd(grid + m * RZ + j * g.Nz + i, make_float2(fx_value(hr, lr) * f, fx_value(hi, li) * f));
  }
}

// rho of one particle straight into the global grid (any Nm; the moving window's injection).
__device__ __forceinline__ void deposit_rho_global(const GeomF& g, float2* rho, const float* invV, float q, int iz,
                                                   float fz, float x, float y, float w) {
  float r, c, s;
  polar_rcp(x, y, r, c, s);
  const RadW rw = radial_nodes(r, g.Nr);
  const int RZ = g.Nr * g.Nz;
  for (int row = 0; row < 2; ++row) {
    const int i = row ? (iz + 1 == g.Nz ? 0 : iz + 1) : iz;
    const float wz = row ? fz : 1.f - fz;
    for (int node = 0; node < 2; ++node) {
      const float sP = wz * (node ? rw.b : rw.aP), sM = wz * (node ? rw.b : rw.aM);
      if (sP == 0.f && sM == 0.f) continue;
      const int j = rw.jb + node;
      float pr = q * w, pi = 0.f;
      for (int m = 0; m < g.Nm; ++m) {
        const float f = (class_p(true, m) ? sP : sM) * invV[j];
        atomicAdd(rho + m * RZ + j * g.Nz + i, make_float2(pr * f, pi * f));
        const float nr = pr * c - pi * s;
        pi = pr * s + pi * c;
        pr = nr;
      }
    }
  }
}

__global__ void k_inv_volume_f(float* invV, int Nr, double dr, double dz) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < Nr) invV[j] = (float)(1.0 / (2.0 * kPi * ((j + 0.5) * dr) * dr * dz));
}

template <bool WIN>
__global__ void k_keys_f32(const PartsF p, int64_t np, GeomF g, int32_t* keys, int32_t* count, int32_t* err) {
  const int ncell = g.Nz * g.Nr;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (WIN) {
      const bool inactive = p.w[i] == 0.f;
      count_inactive(count, tail_key(ncell, i), inactive);
      if (inactive) {
        keys[i] = tail_key(ncell, i);
        continue;
      }
    }
    float x, y;
    pos_cells(p, i, x, y);
    const float r = sqrtf(__fadd_rn(__fmul_rn(x, x), __fmul_rn(y, y)));
    float fr = floorf(r);
    int iz = p.iz[i];
    if (!(fr == fr) || isinf(fr) || iz < 0 || iz >= g.Nz) {
      atomicOr(err, kErrNumeric);
      fr = 0.f;
      iz = 0;
    }
    const int ir = (int)fminf(fmaxf(fr, 0.f), (float)(g.Nr - 1));
    const int key = iz * g.Nr + ir;
    keys[i] = key;
    atomicAdd(count + key, 1);
  }
}

// dst[i] = src[perm[i]] for the 13 arrays; four particles per thread, all loads issued
// before the stores (the gathered reads are latency-bound).
template <bool WIN>
__global__ void k_permute_f32(const PartsF src, PartsF dst, const int32_t* __restrict__ perm, int64_t np,
                              int32_t* slot) {
  constexpr int U = 4;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i0 < np; i0 += U * stride) {
    int32_t k[U];
    bool ok[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int64_t i = i0 + u * stride;
      ok[u] = i < np;
      k[u] = ok[u] ? perm[i] : 0;
    }
    int32_t iz[U], ixy[U], id[U];
    float fz[U], fx[U], fy[U], ux[U], uy[U], uz[U], uxl[U], uyl[U], uzl[U], w[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int32_t j = k[u];
      iz[u] = src.iz[j]; fz[u] = src.fz[j]; ixy[u] = src.ixy[j]; fx[u] = src.fx[j]; fy[u] = src.fy[j];
      ux[u] = src.ux[j]; uy[u] = src.uy[j]; uz[u] = src.uz[j];
      uxl[u] = src.uxl[j]; uyl[u] = src.uyl[j]; uzl[u] = src.uzl[j];
      w[u] = src.w[j]; id[u] = src.id[j];
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      if (!ok[u]) continue;
      const int64_t i = i0 + u * stride;
      dst.iz[i] = iz[u]; dst.fz[i] = fz[u]; dst.ixy[i] = ixy[u]; dst.fx[i] = fx[u]; dst.fy[i] = fy[u];
      dst.ux[i] = ux[u]; dst.uy[i] = uy[u]; dst.uz[i] = uz[u];
      dst.uxl[i] = uxl[u]; dst.uyl[i] = uyl[u]; dst.uzl[i] = uzl[u];
      dst.w[i] = w[u]; dst.id[i] = id[u];
      if (WIN && w[u] == 0.f) slot[id[u]] = (int32_t)i;   // moving window: inactive slot by id
    }
  }
}

// One CTA per chunk of `chunk` consecutive (cell-sorted) particles.  Threads per CTA of the
// band kernels: one band (up to kBandBudget bytes) per CTA, two CTAs per SM; 512 threads x
// 64 registers x 2 CTAs fill the register file.
constexpr int kBandThreads = 512;

// rho and/or J of the particles with id in [id_lo, id_hi) at their current positions
// (the stage call pic_deposit, the ion background, the beams' initial fields).
// KIND 1: rho (band of 1 component), 2: J (3), 3: both (4, rho first).
template <int NM, int KIND>
__global__ void __launch_bounds__(kBandThreads, 2) k_deposit_f32(const PartsF p, int64_t np, GeomF g, DepArgsF a,
                                                                   const float* invV, int32_t* err, BandArgs ba) {
  constexpr bool DO_RHO = KIND & 1, DO_J = (KIND & 2) != 0;
  constexpr int NC = (DO_RHO ? 1 : 0) + (DO_J ? 3 : 0);
  extern __shared__ __align__(16) int32_t band_smem[];
  __shared__ ChunkStats stats_slot;
  const float c_light = (float)kC;
  const int64_t b0 = blockIdx.x * ba.chunk;
  if (b0 >= np) return;
  const int64_t b1 = b0 + ba.chunk < np ? b0 + ba.chunk : np;
  BandF band{nullptr, 0, 0, 0, 0, 1, 0, 1.f, 1.f};
  if (ba.tz > 0) {
    const ChunkStats cs = chunk_stats(p, g, b0, b1, &stats_slot, err);
    const float qw = fabsf(a.q) * __uint_as_float(cs.wmax_bits);
    if (cs.wmax_bits != 0u)   // a chunk of inactive particles deposits nothing: no band
      band = make_band(band_smem, p.iz[b0], p.iz[b1 - 1], g, ba.tz, band_node_words(NM, NC), cs, ba.jw_max,
                       ba.jmargin, ba.lg_chunk, qw * c_light, qw);
  }
  band_zero(band);
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const int32_t id = p.id[i];
    if (id < a.id_lo || id >= a.id_hi) continue;
    const float wt = p.w[i];
    if (wt == 0.f) continue;   // inactive particles add nothing
    float x, y;
    pos_cells(p, i, x, y);
    const float fz = p.fz[i];
    const int iz = p.iz[i];
    if (!isfinite(x) || !isfinite(y) || !isfinite(fz) || iz < 0 || iz >= g.Nz) {
      atomicOr(err, kErrNumeric);
      continue;
    }
    float vx = 0.f, vy = 0.f, vz = 0.f;
    if (DO_J) {
      const float ux = p.ux[i] + p.uxl[i], uy = p.uy[i] + p.uyl[i], uz = p.uz[i] + p.uzl[i];
      const float ig = c_light * rsqrtf(1.f + ux * ux + uy * uy + uz * uz);
      vx = ux * ig; vy = uy * ig; vz = uz * ig;
    }
    deposit_nodes<NM, NC, DO_RHO, DO_J>(band, g, a, invV, iz, fz, x, y, wt, vx, vy, vz);
  }
  __syncthreads();
  band_flush<NM, NC, DO_RHO>(band, g, a.rho, a.J, invV);
}

// Advance (iz, fz) by dfz cells, periodic in iz.
__device__ __forceinline__ void advance_z(int& iz, float& fz, float dfz, int Nz) {
  fz += dfz;
  const float k = floorf(fz);
  fz -= k;
  if (fz >= 1.f) { fz -= 1.f; iz += 1; }   // rounding of fz - k up to 1
  iz += (int)k;
  iz %= Nz;
  if (iz < 0) iz += Nz;
}

// a2 + a3 (+ a4 J at x^{n+1/2}) in float: gather with mode sum from the node-major copy of
// E and B, Boris push of u/c, two half moves (z in cell units), specular reflection at
// r >= R.  One CTA per chunk of `chunk` consecutive (cell-sorted) particles; with fuse and
// tz > 0 the J deposit accumulates into a band of z rows from one row below the chunk's
// first cell (a half step moves a particle by at most half a cell at c dt <= dz).
// RHO: also deposit rho^{n+1} at x^{n+1} (band component 0; J in components 1..3, which is
// the order of the deposit grids, so one flush writes all four).
template <int NM, bool WIN, bool RHO>
__global__ void __launch_bounds__(kBandThreads, 2) k_gather_push_f32(PartsF p, int64_t np, GeomF g,
                                  const float2* __restrict__ ebn, float kq, float kqc, float chdt_dr,
                                  float chdt_dz, DepArgsF dep, const float* invV, int fuse, int32_t* err,
                                  BandArgs ba, WinArgs wa) {
  constexpr int NC = RHO ? 4 : 3;
  extern __shared__ __align__(16) int32_t band_smem[];
  __shared__ ChunkStats stats_slot;
  const float c_light = (float)kC;
  const int64_t b0 = blockIdx.x * ba.chunk;
  if (b0 >= np) return;
  const int64_t b1 = b0 + ba.chunk < np ? b0 + ba.chunk : np;
  BandF band{nullptr, 0, 0, 0, 0, 1, 0, 1.f, 1.f};
  if (fuse && ba.tz > 0) {
    const ChunkStats cs = chunk_stats(p, g, b0, b1, &stats_slot, err);
    const float qw = fabsf(dep.q) * __uint_as_float(cs.wmax_bits);
    if (cs.wmax_bits != 0u)   // a chunk of inactive particles deposits nothing: no band
      band = make_band(band_smem, p.iz[b0], p.iz[b1 - 1], g, ba.tz, band_node_words(NM, NC), cs, ba.jw_max,
                       ba.jmargin, ba.lg_chunk, qw * c_light, qw);
  }
  band_zero(band);
  __syncthreads();
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const float w = p.w[i];
    if (w == 0.f) continue;   // inactive (moving window): neither pushed nor moved
    const int32_t cells = p.ixy[i];
    int ix = cell_x(cells), iy = cell_y(cells);
    float fx = p.fx[i], fy = p.fy[i], fz = p.fz[i];
    int iz = p.iz[i];
    float x = (float)ix + fx, y = (float)iy + fy;   // cells
    if (!isfinite(x) || !isfinite(y) || !isfinite(fz) || iz < 0 || iz >= g.Nz) {
      atomicOr(err, kErrNumeric);
      continue;
    }
    // window coordinate at x^n in cells (exact for the cells near the back edge)
    float zeta_old = 0.f;
    if (WIN) {
      int zrel = iz - wa.back_col;
      if (zrel < 0) zrel += g.Nz;
      zeta_old = (float)zrel + fz;
    }
    float r, c, s;
    polar_rcp(x, y, r, c, s);
    float F[6];
    gather_nodes<NM>(ebn, g.Nr, iz, iz + 1 == g.Nz ? 0 : iz + 1, 1.f - fz, fz, radial_nodes(r, g.Nr), c, s, F);
    float uxh = p.ux[i], uyh = p.uy[i], uzh = p.uz[i];
    float uxl = p.uxl[i], uyl = p.uyl[i], uzl = p.uzl[i];
    const float Ex = F[0] * c - F[1] * s, Ey = F[0] * s + F[1] * c, Ez = F[2];
    const float Bx = F[3] * c - F[4] * s, By = F[3] * s + F[4] * c, Bz = F[5];
    // Boris on u/c: u- = u + kq E, t = kqc B / gamma-, kq = q dt/(2 m c), kqc = q dt/(2 m).
    // The increments are formed in float from float values of u; the sums are kept as pairs.
    const float ex = kq * Ex, ey = kq * Ey, ez = kq * Ez;
    ff_add(uxh, uxl, ex); ff_add(uyh, uyl, ey); ff_add(uzh, uzl, ez);   // u-
    const float umx = uxh + uxl, umy = uyh + uyl, umz = uzh + uzl;
    const float igm = rsqrtf(1.f + umx * umx + umy * umy + umz * umz);
    const float tx = kqc * Bx * igm, ty = kqc * By * igm, tz = kqc * Bz * igm;
    const float upx = umx + (umy * tz - umz * ty);
    const float upy = umy + (umz * tx - umx * tz);
    const float upz = umz + (umx * ty - umy * tx);
    const float f = 2.f / (1.f + tx * tx + ty * ty + tz * tz);
    const float sx = f * tx, sy = f * ty, sz = f * tz;
    ff_add(uxh, uxl, upy * sz - upz * sy);   // u+ = u- + u' x s
    ff_add(uyh, uyl, upz * sx - upx * sz);
    ff_add(uzh, uzl, upx * sy - upy * sx);
    ff_add(uxh, uxl, ex); ff_add(uyh, uyl, ey); ff_add(uzh, uzl, ez);   // u^{n+1/2}
    const float ux = uxh + uxl, uy = uyh + uyl, uz = uzh + uzl;
    const float ig = rsqrtf(1.f + ux * ux + uy * uy + uz * uz);
    const float bx = ux * ig, by = uy * ig, bz = uz * ig;   // v / c
    const float dzc = bz * chdt_dz;                          // half move in cells
    advance_cell(ix, fx, bx * chdt_dr);
    advance_cell(iy, fy, by * chdt_dr);
    advance_z(iz, fz, dzc, g.Nz);
    if (fuse)
      deposit_nodes<NM, NC, false, true>(band, g, dep, invV, iz, fz, (float)ix + fx, (float)iy + fy, w,
                                         bx * c_light, by * c_light, bz * c_light);
    advance_cell(ix, fx, bx * chdt_dr);
    advance_cell(iy, fy, by * chdt_dr);
    advance_z(iz, fz, dzc, g.Nz);
    x = (float)ix + fx;
    y = (float)iy + fy;
    const float r1 = sqrtf(x * x + y * y);
    if (r1 >= (float)g.Nr) {   // specular reflection at r = R
      const float cx = x / r1, cy = y / r1;
      const float fr = (2.f * (float)g.Nr - r1) / r1;
      const float ur = ux * cx + uy * cy;
      ff_add(uxh, uxl, -2.f * ur * cx);
      ff_add(uyh, uyl, -2.f * ur * cy);
      x *= fr;
      y *= fr;
      const float kx = floorf(x), ky = floorf(y);
      ix = (int)kx; fx = x - kx;
      iy = (int)ky; fy = y - ky;
      if (fx >= 1.f) { fx = 0.f; ix += 1; }
      if (fy >= 1.f) { fy = 0.f; iy += 1; }
    }
    bool removed = false;
    if (WIN && (zeta_old + dzc) + dzc - (wa.shift ? 1.f : 0.f) < 0.f) {
      p.w[i] = 0.f;   // left through the back edge: inactive from now on
      uxh = uyh = uzh = 0.f;
      uxl = uyl = uzl = 0.f;
      win_mark(wa, p.id[i], i);
      removed = true;
    }
    p.ixy[i] = pack_cells(ix, iy); p.fx[i] = fx; p.fy[i] = fy; p.fz[i] = fz; p.iz[i] = iz;
    p.ux[i] = uxh; p.uy[i] = uyh; p.uz[i] = uzh;
    p.uxl[i] = uxl; p.uyl[i] = uyl; p.uzl[i] = uzl;
    if (RHO && fuse && !removed)   // rho^{n+1} at x^{n+1} (a removed particle has left)
      deposit_nodes<NM, NC, true, false>(band, g, dep, invV, iz, fz, x, y, w, 0.f, 0.f, 0.f);
  }
  __syncthreads();
  band_flush<NM, NC, RHO>(band, g, dep.rho, dep.J, invV);
}

// float64 SoA (x y z ux uy uz w) <-> FP32 cell-relative particles
__device__ __forceinline__ void split_cell(double u, int& cell, float& f) {
  const double fl = floor(u);
  f = (float)(u - fl);
  long long c = (long long)fl;
  if (f >= 1.f) { f = 0.f; c += 1; }
  cell = (int)c;
}

__device__ __forceinline__ void split_pair(double u, float& h, float& l) {
  h = (float)u;
  l = (float)(u - (double)h);
}

// Cells and fractions from x / dr etc. taken as x * (1/dr) (reciprocals from the host): a
// float64 division is a long sequence on GB300's float64 units, and the product differs by at
// most one float64 ulp, far below the float fraction's resolution.
__global__ void k_p64_to_p32(const double* __restrict__ st, int64_t cap, const int32_t* __restrict__ id_in,
                             PartsF p, int64_t np, int Nz, double inv_dz, double inv_dr) {
  constexpr double inv_c = 1.0 / kC;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    int iz, ix, iy;
    float fz, fx, fy;
    split_cell(st[2 * cap + i] * inv_dz, iz, fz);
    iz %= Nz;
    if (iz < 0) iz += Nz;
    split_cell(st[i] * inv_dr, ix, fx);
    split_cell(st[cap + i] * inv_dr, iy, fy);
    p.iz[i] = iz;
    p.fz[i] = fz;
    p.ixy[i] = pack_cells(ix, iy);
    p.fx[i] = fx;
    p.fy[i] = fy;
    split_pair(st[3 * cap + i] * inv_c, p.ux[i], p.uxl[i]);
    split_pair(st[4 * cap + i] * inv_c, p.uy[i], p.uyl[i]);
    split_pair(st[5 * cap + i] * inv_c, p.uz[i], p.uzl[i]);
    p.w[i] = (float)st[6 * cap + i];
    p.id[i] = id_in[i];
  }
}

__global__ void k_p32_to_p64(const PartsF p, int64_t np, double* __restrict__ st, int64_t cap,
                             int32_t* __restrict__ id_out, double dz, double dr) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t c = p.ixy[i];
    st[i] = ((double)cell_x(c) + (double)p.fx[i]) * dr;
    st[cap + i] = ((double)cell_y(c) + (double)p.fy[i]) * dr;
    st[2 * cap + i] = ((double)p.iz[i] + (double)p.fz[i]) * dz;
    st[3 * cap + i] = ((double)p.ux[i] + (double)p.uxl[i]) * kC;
    st[4 * cap + i] = ((double)p.uy[i] + (double)p.uyl[i]) * kC;
    st[5 * cap + i] = ((double)p.uz[i] + (double)p.uzl[i]) * kC;
    st[6 * cap + i] = p.w[i];
    if (id_out) id_out[i] = p.id[i];
  }
}

// ------------------------------------------------------------------ a10: diagnostics
// Particle accessors: float64 particles as stored, or FP32 particles widened to float64.
// z is measured from z0 (the moving window's back edge, 0 without a window), mod L.
struct Acc64 {
  Parts p;
  double z0, L;
  __device__ void get(int64_t i, double& x, double& y, double& z, double& ux, double& uy, double& uz,
                      double& w) const {
    x = p.x[i]; y = p.y[i]; z = p.z[i]; ux = p.ux[i]; uy = p.uy[i]; uz = p.uz[i]; w = p.w[i];
    if (z0 != 0.0) {
      z -= z0;
      if (z < 0.0) z += L;
    }
  }
  __device__ int32_t id(int64_t i) const { return p.id[i]; }
};
struct Acc32 {
  PartsF p;
  double dz, dr;
  int col0, Nz;   // z is measured from column col0 (the window's back column, 0 without one)
  __device__ void get(int64_t i, double& x, double& y, double& z, double& ux, double& uy, double& uz,
                      double& w) const {
    const int32_t c = p.ixy[i];
    x = ((double)cell_x(c) + (double)p.fx[i]) * dr;
    y = ((double)cell_y(c) + (double)p.fy[i]) * dr;
    int iz = p.iz[i] - col0;
    if (iz < 0) iz += Nz;
    z = ((double)iz + (double)p.fz[i]) * dz;
    ux = ((double)p.ux[i] + (double)p.uxl[i]) * kC;
    uy = ((double)p.uy[i] + (double)p.uyl[i]) * kC;
    uz = ((double)p.uz[i] + (double)p.uzl[i]) * kC;
    w = p.w[i];
  }
  __device__ int32_t id(int64_t i) const { return p.id[i]; }
};

// Diagnostics grid: at most kDiagMaxGrid CTAs of kDiagThreads threads.  Sums over the
// particles are formed per CTA, stored as per-CTA partials and added in CTA order by the
// last CTA to finish (an integer ticket): float64 atomics from every CTA onto the same few
// addresses serialise in L2, and the fixed order makes the results reproducible.
constexpr int kDiagMaxGrid = 8 * 152;

// The selected particles (id in [lo, hi)) of one diagnostics call, compacted in array order
// as float64 x, y, z, ux, uy, w, gamma (7 arrays; z is replaced by the slice index, or -1
// outside the slice span, in the first slice pass).  The passes over the compacted set
// spread the float64 work of a beam (a few CTAs' worth of the cell-sorted arrays) over the
// whole GPU; float64 arithmetic is slow on GB300.
struct DiagC {
  double* v[7];
};

// Header of the accumulator block: [0..7] pass-1 sums (w, w x, w y, w z, w ux, w uy,
// w gamma, count), [16..20] means, [32..38] pass-2 sums, [48] slice start, [49] slice span,
// [50] slices, [51] status (0 ok, 1 no weight, 2 sigma_z = 0, 3 too many slices),
// [52] non-empty slices, [53] sum of the slice spreads, [56] compacted count (uint64),
// [57], [58] tickets of the two reductions (uint32).  After the header, the slice sums,
// the inverse cell volumes, then the per-CTA partials and counts (diag_parts).
enum {
  kDiagMean = 16, kDiagC2 = 32, kDiagZ0 = 48, kDiagSpan = 49, kDiagNs = 50, kDiagStatus = 51, kDiagNe = 52,
  kDiagSigSum = 53, kDiagCount = 56, kDiagTicket = 57
};

struct DiagParts {
  double* p1;     // [kDiagMaxGrid][8]
  double* p2;     // [kDiagMaxGrid][8]
  int64_t* cnt;   // [kDiagMaxGrid]
};

__device__ __forceinline__ int64_t diag_count(const double* acc) {
  return (int64_t)*reinterpret_cast<const unsigned long long*>(acc + kDiagCount);
}

// CTA sums of K per-thread values into part[blockIdx.x][0..K); the last CTA adds the
// partials of all CTAs in CTA order into out[0..K).  Every CTA of the grid calls it.
// active: this thread added something (a warp without one skips its float64 shuffle sums).
template <int K>
__device__ void block_partials(const double (&v)[K], bool active, double* part, unsigned* ticket, double* out) {
  static_assert(K <= kDiagThreads / 32, "one warp per value in the final sum");
  __shared__ double wsum[kDiagThreads / 32][K];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const bool any = __any_sync(0xffffffffu, active);
#pragma unroll
  for (int k = 0; k < K; ++k) {
    const double t = any ? warp_sum(v[k]) : 0.0;
    if (lane == 0) wsum[warp][k] = t;
  }
  __syncthreads();
  if (threadIdx.x < K) {
    double t = 0.0;
    for (int w = 0; w < kDiagThreads / 32; ++w) t += wsum[w][threadIdx.x];
    part[blockIdx.x * 8 + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (warp < K) {
    double t = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) t += __ldcg(part + b * 8 + warp);
    t = warp_sum(t);
    if (lane == 0) out[warp] = t;
  }
}

// CTA b of the selection passes walks particles [b C, (b+1) C), C = ceil(np / grid) rounded
// up to whole iterations of the CTA.
__device__ __forceinline__ void diag_chunk(int64_t np, int64_t& b0, int64_t& b1) {
  const int64_t per = ((np + gridDim.x - 1) / gridDim.x + kDiagThreads - 1) / kDiagThreads * kDiagThreads;
  b0 = blockIdx.x * per;
  b1 = min(np, b0 + per);
}

// pass 0: number of selected particles of each CTA's chunk.
template <class A>
__global__ void __launch_bounds__(kDiagThreads) k_diag_count(const A a, int64_t np, int32_t lo, int32_t hi,
                                                              DiagParts dp) {
  __shared__ int32_t wc[kDiagThreads / 32];
  int64_t b0, b1;
  diag_chunk(np, b0, b1);
  int32_t c = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) {
    const int32_t id = a.id(i);
    c += (id >= lo && id < hi) ? 1 : 0;
  }
  c = __reduce_add_sync(0xffffffffu, c);
  if ((threadIdx.x & 31) == 0) wc[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kDiagThreads / 32; ++w) t += wc[w];
    dp.cnt[blockIdx.x] = t;
  }
}

// pass 1: compact the selected particles in array order (each CTA's offset is the sum of
// the counts of the CTAs before it) and sum w, w x, w y, w z, w ux, w uy, w gamma, count.
template <class A>
__global__ void __launch_bounds__(kDiagThreads) k_diag_select(const A a, int64_t np, int32_t lo, int32_t hi,
                                                               DiagC c, DiagParts dp, double* acc) {
  __shared__ int64_t wred[kDiagThreads / 32];
  __shared__ int32_t wbase[kDiagThreads / 32];
  __shared__ int64_t base;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // offset of this CTA: sum of the counts of CTAs 0 .. blockIdx.x - 1
  int64_t s = 0;
  for (int b = threadIdx.x; b < (int)blockIdx.x; b += blockDim.x) s += dp.cnt[b];
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  if (lane == 0) wred[warp] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kDiagThreads / 32; ++w) t += wred[w];
    base = t;
    if (blockIdx.x == gridDim.x - 1)   // the total, for the passes over the compacted set
      *reinterpret_cast<unsigned long long*>(acc + kDiagCount) = (unsigned long long)(t + dp.cnt[blockIdx.x]);
  }
  __syncthreads();
  int64_t b0, b1;
  diag_chunk(np, b0, b1);
  double v[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  for (int64_t it = b0; it < b1; it += blockDim.x) {
    const int64_t i = it + threadIdx.x;
    bool sel = false;
    if (i < b1) {
      const int32_t id = a.id(i);
      sel = id >= lo && id < hi;
    }
    const unsigned m = __ballot_sync(0xffffffffu, sel);
    if (lane == 0) wbase[warp] = __popc(m);
    __syncthreads();
    if (threadIdx.x == 0) {
      int32_t t = 0;
      for (int w = 0; w < kDiagThreads / 32; ++w) {
        const int32_t k = wbase[w];
        wbase[w] = t;
        t += k;
      }
      wred[0] = t;
    }
    __syncthreads();
    if (sel) {
      const int64_t slot = base + wbase[warp] + __popc(m & ((1u << lane) - 1u));
      double x, y, z, ux, uy, uz, w;
      a.get(i, x, y, z, ux, uy, uz, w);
      const double gam = sqrt(1.0 + (ux * ux + uy * uy + uz * uz) * kInvC2);
      c.v[0][slot] = x; c.v[1][slot] = y; c.v[2][slot] = z;
      c.v[3][slot] = ux; c.v[4][slot] = uy; c.v[5][slot] = w; c.v[6][slot] = gam;
      v[0] += w; v[1] += w * x; v[2] += w * y; v[3] += w * z;
      v[4] += w * ux; v[5] += w * uy; v[6] += w * gam; v[7] += 1.0;
    }
    __syncthreads();   // all reads of wbase and wred[0] done before thread 0 rewrites them
    if (threadIdx.x == 0) base += wred[0];
  }
  block_partials<8>(v, v[7] != 0.0, dp.p1, reinterpret_cast<unsigned*>(acc + kDiagTicket), acc);
}

// pass 2: means (thread 0 of each CTA; CTA 0 stores them and the status), then the centred
// second moments w dx^2, w dux^2, w dx dux, (y), w dz^2 over the compacted particles.
__global__ void __launch_bounds__(kDiagThreads) k_diag_central(DiagC c, DiagParts dp, double* acc) {
  __shared__ double mean[5];
  __shared__ int ok;
  if (threadIdx.x == 0) {
    ok = acc[7] != 0.0 && acc[0] > 0.0;
    if (ok)
      for (int k = 0; k < 5; ++k) mean[k] = acc[1 + k] / acc[0];
    if (blockIdx.x == 0) {
      if (!ok) acc[kDiagStatus] = 1.0;
      else
        for (int k = 0; k < 5; ++k) acc[kDiagMean + k] = mean[k];
    }
  }
  __syncthreads();
  if (!ok) return;   // every CTA: no reduction follows
  const int64_t n = diag_count(acc);
  double v[7] = {0, 0, 0, 0, 0, 0, 0};
  const bool active = blockIdx.x * (int64_t)blockDim.x + threadIdx.x < n;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double w = c.v[5][i];
    const double dx = c.v[0][i] - mean[0], dy = c.v[1][i] - mean[1], dz = c.v[2][i] - mean[2];
    const double dux = c.v[3][i] - mean[3], duy = c.v[4][i] - mean[4];
    v[0] += w * (dx * dx); v[1] += w * (dux * dux); v[2] += w * (dx * dux);
    v[3] += w * (dy * dy); v[4] += w * (duy * duy); v[5] += w * (dy * duy);
    v[6] += w * (dz * dz);
  }
  block_partials<7>(v, active, dp.p2, reinterpret_cast<unsigned*>(acc + kDiagTicket) + 2, acc + kDiagC2);
}

// Slice passes: one compacted particle per thread and iteration; each warp adds each run of
// lanes with equal slices with one atomic from the run's first lane (a segmented sum over
// the warp).  The compacted order keeps the cell order, so a warp's 32 consecutive
// particles usually fall in one or two slices.
__device__ __forceinline__ unsigned run_heads(int key) {
  const int lane = threadIdx.x & 31;
  const int prev = __shfl_up_sync(0xffffffffu, key, 1);
  return __ballot_sync(0xffffffffu, lane == 0 || key != prev);
}

// Sum of v over this lane and the following lanes of its run (heads: first lanes of the
// runs); the first lane of a run receives the run's total.
__device__ __forceinline__ double run_sum(double v, unsigned heads) {
  const int lane = threadIdx.x & 31;
  const unsigned after = heads & ~((2u << lane) - 1u);   // run starts after this lane
  const int end = after ? __ffs(after) - 1 : 32;
  for (int d = 1; d < 32; d <<= 1) {
    const double o = __shfl_down_sync(0xffffffffu, v, d);
    if (lane + d < end) v += o;
  }
  return v;
}

// stage 0: slice layout from sigma_z (thread 0 of each CTA; CTA 0 stores it and the
// status), the slice index of each particle, per-slice sum w and sum w gamma.
__global__ void __launch_bounds__(kDiagThreads) k_diag_slices0(DiagC c, double* acc, double slen, int max_slices,
                                                                double* sw, double* sg) {
  __shared__ double z0, span;
  __shared__ int ns, st;
  if (threadIdx.x == 0) {
    st = (int)acc[kDiagStatus];
    if (st == 0) {
      const double sz = sqrt(acc[kDiagC2 + 6] / acc[0]);
      if (!(sz > 0.0)) {
        st = 2;
      } else {
        span = 6.0 * sz;
        const double nsd = ceil(span / slen);
        z0 = acc[kDiagMean + 2] - 3.0 * sz;
        ns = (int)fmin(nsd, (double)max_slices);
        if (nsd > max_slices) st = 3;
        if (blockIdx.x == 0) {
          acc[kDiagZ0] = z0;
          acc[kDiagSpan] = span;
          acc[kDiagNs] = nsd;
        }
      }
      if (blockIdx.x == 0) acc[kDiagStatus] = (double)st;
    }
  }
  __syncthreads();
  if (st != 0) return;
  const int64_t n = diag_count(acc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const int64_t i = b + (threadIdx.x & 31);   // the warp's lanes: 32 consecutive particles
    int k = -1;
    double w = 0.0, wg = 0.0;
    if (i < n) {
      const double d = c.v[2][i] - z0;
      if (d >= 0.0 && d < span) {
        k = (int)floor(d / slen);
        if (k > ns - 1) k = ns - 1;
        w = c.v[5][i];
        wg = w * c.v[6][i];
      }
      c.v[2][i] = (double)k;
    }
    const unsigned heads = run_heads(k);
    w = run_sum(w, heads);
    wg = run_sum(wg, heads);
    if (k >= 0 && ((heads >> (threadIdx.x & 31)) & 1u)) {
      atomicAdd(sw + k, w);
      atomicAdd(sg + k, wg);
    }
  }
}

// stage 1: per-slice sum w (gamma - gbar_s)^2, gbar_s = sum w gamma / sum w of the slice.
__global__ void __launch_bounds__(kDiagThreads) k_diag_slices1(DiagC c, const double* acc, const double* sw,
                                                                const double* sg, double* sv) {
  if (acc[kDiagStatus] != 0.0) return;
  const int64_t n = diag_count(acc);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t b = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); b < n; b += stride) {
    const int64_t i = b + (threadIdx.x & 31);
    int k = -1;
    double v = 0.0;
    if (i < n) {
      k = (int)c.v[2][i];
      if (k >= 0 && sw[k] > 0.0) {   // a slice of zero weight has no spread
        const double dg = c.v[6][i] - sg[k] / sw[k];
        v = c.v[5][i] * (dg * dg);
      }
    }
    const unsigned heads = run_heads(k);
    v = run_sum(v, heads);
    if (k >= 0 && ((heads >> (threadIdx.x & 31)) & 1u)) atomicAdd(sv + k, v);
  }
}

// Per-slice std of gamma of the non-empty slices, in slice order, into out[0 .. ne) (one CTA
// of 1024 threads; ranks by a block scan); ne and the sum of the spreads into the header.
__global__ void __launch_bounds__(1024) k_diag_slice_compact(double* hdr, const double* sw, const double* sv,
                                                              double* out) {
  __shared__ double part[32];
  if (hdr[kDiagStatus] != 0.0) return;
  const int ns = (int)hdr[kDiagNs];
  int32_t base = 0;
  double sum = 0.0;
  for (int k0 = 0; k0 < ns; k0 += 1024) {
    const int k = k0 + threadIdx.x;
    const bool ne = k < ns && sw[k] > 0.0;
    int32_t tot;
    const int32_t pos = base + block_exclusive_scan(ne ? 1 : 0, &tot);
    if (ne) {
      const double sg = sqrt(sv[k] / sw[k]);
      out[pos] = sg;
      sum += sg;
    }
    base += tot;
  }
  sum = warp_sum(sum);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = sum;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 32; ++w) t += part[w];
    hdr[kDiagNe] = (double)base;
    hdr[kDiagSigSum] = t;
  }
}

inline int pgrid(int64_t n) {
  int64_t b = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, 152 * 16));
}

// Compacted-particle storage of the diagnostics: the staging area (mixed forms) or the
// particle buffer that is not current (FP64 form); both are free between cycles.
DiagC diag_storage(Sim* s) {
  DiagC c;
  const size_t cap = (size_t)s->cfg.np_capacity;
  for (int k = 0; k < 7; ++k)
    c.v[k] = s->cfg.precision != PIC_FP64 ? s->at<double>(s->lay.stage64) + k * cap
                                          : s->at<double>(s->lay.part[1 - s->cur][k]);
  return c;
}

constexpr size_t kDiagPartsDoubles = 2 * 8 * (size_t)kDiagMaxGrid + kDiagMaxGrid;

DiagParts diag_parts(Sim* s) {
  double* p = s->at<double>(s->lay.diag_acc) + 64 + 3 * (size_t)kMaxSlices + kMaxNr;
  return DiagParts{p, p + 8 * kDiagMaxGrid, reinterpret_cast<int64_t*>(p + 16 * kDiagMaxGrid)};
}

// The passes chain on the device; one copy of the header and the requested slice values
// and one synchronisation at the end.
template <class A>
pic_status run_diag(Sim* s, const A& acc_p, int32_t lo, int32_t hi, pic_diag* out, double* slice_sigma,
                    int32_t max_slices) {
  const int64_t np = s->np;
  double* acc = s->at<double>(s->lay.diag_acc);
  double* sw = acc + 64;
  double* sg = sw + kMaxSlices;
  double* sv = sg + kMaxSlices;
  const DiagC c = diag_storage(s);
  const DiagParts dp = diag_parts(s);
  PIC_CUDA(cudaMemsetAsync(acc, 0, 64 * sizeof(double), s->stream));
  PIC_CUDA(cudaMemsetAsync(sw, 0, 3 * sizeof(double) * kMaxSlices, s->stream));
  const int grid = std::min(pgrid(np), kDiagMaxGrid);
  if (np > 0) {
    k_diag_count<A><<<grid, kDiagThreads, 0, s->stream>>>(acc_p, np, lo, hi, dp);
    PIC_LAUNCHED(s);
    k_diag_select<A><<<grid, kDiagThreads, 0, s->stream>>>(acc_p, np, lo, hi, c, dp, acc);
    PIC_LAUNCHED(s);
  }
  // one CTA per SM: a few compacted particles per thread amortise the CTA's float64 sums
  k_diag_central<<<std::min(grid, 152), kDiagThreads, 0, s->stream>>>(c, dp, acc);
  PIC_LAUNCHED(s);
  k_diag_slices0<<<grid, kDiagThreads, 0, s->stream>>>(c, acc, kSliceLen, kMaxSlices, sw, sg);
  PIC_LAUNCHED(s);
  k_diag_slices1<<<grid, kDiagThreads, 0, s->stream>>>(c, acc, sw, sg, sv);
  PIC_LAUNCHED(s);
  k_diag_slice_compact<<<1, 1024, 0, s->stream>>>(acc, sw, sv, sg);   // sg is free after stage 1
  PIC_LAUNCHED(s);
  if (!s->diag_host) PIC_CUDA(cudaMallocHost(&s->diag_host, (64 + (size_t)kMaxSlices) * sizeof(double)));
  double* h = s->diag_host;
  const double* sig = h + 64;
  const int32_t n_copy = slice_sigma ? std::min<int32_t>(std::max<int32_t>(max_slices, 0), kMaxSlices) : 0;
  PIC_CUDA(cudaMemcpyAsync(h, acc, 64 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  if (n_copy > 0)
    PIC_CUDA(cudaMemcpyAsync(h + 64, sg, n_copy * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
  PIC_CUDA(cudaStreamSynchronize(s->stream));
  *out = pic_diag{};
  out->n_particles = (int32_t)h[7];
  out->W = h[0];
  const int status = (int)h[kDiagStatus];
  if (status == 1) return PIC_OK;
  out->x_mean = h[kDiagMean]; out->y_mean = h[kDiagMean + 1]; out->z_mean = h[kDiagMean + 2];
  out->gamma_mean = h[6] / h[0];
  const double W = h[0];
  const double* c2 = h + kDiagC2;
  const double xx = c2[0] / W, uu = c2[1] / W, xu = c2[2] / W;
  const double yy = c2[3] / W, vv = c2[4] / W, yv = c2[5] / W;
  out->emit_nx = std::sqrt(std::max(xx * uu - xu * xu, 0.0)) / kC;
  out->emit_ny = std::sqrt(std::max(yy * vv - yv * yv, 0.0)) / kC;
  out->sigma_z = std::sqrt(c2[6] / W);
  if (status == 2) return PIC_OK;
  if (status == 3) {
    set_error("diagnostics: %g slices exceed the maximum %d", h[kDiagNs], kMaxSlices);
    return PIC_ERR_ARG;
  }
  const int ne = (int)h[kDiagNe];
  for (int k = 0; k < ne && k < n_copy; ++k) slice_sigma[k] = sig[k];
  out->n_slices = ne;
  out->sigma_gamma_mean = ne ? h[kDiagSigSum] / ne : 0.0;
  return PIC_OK;
}

// ------------------------------------------------------------------ moving window
// Template of the plasma, by id (ids < n_tpl): FP64 form x, y, z, w; mixed form the
// cell-relative fields iz, fz, ixy, fx, fy and w.  Both fit in 32 bytes per particle.
struct WinTpl {
  double* x; double* y; double* z; double* w;
};
struct WinTplF {
  int32_t* iz; float* fz; int32_t* ixy; float* fx; float* fy; float* w;
};

WinTpl win_tpl(const Sim* s) {
  double* b = reinterpret_cast<double*>(s->win.ws + s->win.tpl);
  const int64_t n = s->win.n_tpl;
  return WinTpl{b, b + n, b + 2 * n, b + 3 * n};
}
WinTplF win_tplf(const Sim* s) {
  char* b = s->win.ws + s->win.tpl;
  const size_t n4 = 4 * (size_t)s->win.n_tpl;
  return WinTplF{reinterpret_cast<int32_t*>(b), reinterpret_cast<float*>(b + n4),
                 reinterpret_cast<int32_t*>(b + 2 * n4), reinterpret_cast<float*>(b + 3 * n4),
                 reinterpret_cast<float*>(b + 4 * n4), reinterpret_cast<float*>(b + 5 * n4)};
}

// Reserve particle k: id id0 + k, inactive, at the centre of cell (k mod Nz, (k div Nz) mod Nr)
// on the x axis.
__global__ void k_win_reserve(Parts p, int64_t first, int64_t n, int32_t id0, int Nz, int Nr, double dz,
                              double dr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = first + k;
    p.x[i] = ((double)((k / Nz) % Nr) + 0.5) * dr;
    p.y[i] = 0.0;
    p.z[i] = ((double)(k % Nz) + 0.5) * dz;
    p.ux[i] = 0.0; p.uy[i] = 0.0; p.uz[i] = 0.0; p.w[i] = 0.0;
    p.id[i] = id0 + (int32_t)k;
  }
}

__global__ void k_win_reserve_f32(PartsF p, int64_t first, int64_t n, int32_t id0, int Nz, int Nr) {
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < n; k += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = first + k;
    p.iz[i] = (int32_t)(k % Nz);
    p.fz[i] = 0.5f;
    p.ixy[i] = pack_cells((int)((k / Nz) % Nr), 0);
    p.fx[i] = 0.5f;
    p.fy[i] = 0.f;
    p.ux[i] = 0.f; p.uy[i] = 0.f; p.uz[i] = 0.f;
    p.uxl[i] = 0.f; p.uyl[i] = 0.f; p.uzl[i] = 0.f;
    p.w[i] = 0.f;
    p.id[i] = id0 + (int32_t)k;
  }
}

// Template by id and the column of each template particle.
__global__ void k_win_template(const Parts p, int64_t np, int64_t n_tpl, WinTpl t, int32_t* col, int Nz,
                               double dz) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t id = p.id[i];
    if (id < 0 || id >= n_tpl) continue;
    const double z = p.z[i];
    t.x[id] = p.x[i]; t.y[id] = p.y[i]; t.z[id] = z; t.w[id] = p.w[i];
    col[id] = (int32_t)fmin(fmax(floor(z / dz), 0.0), (double)(Nz - 1));
  }
}

__global__ void k_win_template_f32(const PartsF p, int64_t np, int64_t n_tpl, WinTplF t, int32_t* col) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    const int32_t id = p.id[i];
    if (id < 0 || id >= n_tpl) continue;
    t.iz[id] = p.iz[i]; t.fz[id] = p.fz[i]; t.ixy[id] = p.ixy[i];
    t.fx[id] = p.fx[i]; t.fy[id] = p.fy[i]; t.w[id] = p.w[i];
    col[id] = p.iz[i];
  }
}

// Injection.  Every inactive particle has flag[id] = 1, slot[id] = its array index and is
// counted in bcnt[id / 1024] (set at set-up and at removal, slots kept current by the
// permute); the ranks of the flagged ids (increasing id) come from the exclusive scan of the
// counts and a scan inside each block.  Injected ids leave the records.
constexpr int kWinBlock = 1024;

// Every inactive particle recorded (window set-up).
template <typename T>
__global__ void k_win_mark_all(const T* __restrict__ w, const int32_t* __restrict__ id, int64_t np, int32_t* flag,
                               int32_t* slot, int32_t* bcnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < np; i += (int64_t)gridDim.x * blockDim.x) {
    if (w[i] == (T)0) {
      const int32_t k = id[i];
      flag[k] = 1;
      slot[k] = (int32_t)i;
      atomicAdd(bcnt + (k >> 10), 1);
    }
  }
}

// One CTA: bstart = exclusive scan of the nb block counts, bstart[nb] = inactive ids in all;
// template particles without a slot are counted as dropped.
__global__ void __launch_bounds__(kWinBlock) k_win_bscan(const int32_t* bcnt, int32_t* bstart, int nb,
                                                          int32_t n_fresh, unsigned long long* dropped) {
  int32_t carry = 0;
  for (int base = 0; base < nb; base += kWinBlock) {
    const int k = base + threadIdx.x;
    const int32_t v = k < nb ? bcnt[k] : 0;
    int32_t tot;
    const int32_t ex = block_exclusive_scan(v, &tot);
    if (k < nb) bstart[k] = carry + ex;
    carry += tot;
  }
  if (threadIdx.x == 0) {
    bstart[nb] = carry;
    if (carry < n_fresh) atomicAdd(dropped, (unsigned long long)(n_fresh - carry));
  }
}

// Rank of id k among the inactive ids (valid where v = 1).  An id that receives a template
// particle (rank < n_fresh) leaves the records.
__device__ __forceinline__ int32_t win_rank(int32_t* flag, int32_t* bcnt, const int32_t* bstart, int64_t n,
                                            int32_t n_fresh, int& v) {
  const int64_t k = blockIdx.x * (int64_t)kWinBlock + threadIdx.x;
  v = k < n ? flag[k] : 0;
  int32_t tot;
  const int32_t r = bstart[blockIdx.x] + block_exclusive_scan(v, &tot);
  if (v && r < n_fresh) {
    flag[k] = 0;
    atomicSub(bcnt + blockIdx.x, 1);
  }
  return r;
}

__global__ void __launch_bounds__(kWinBlock) k_win_inject(int32_t* flag, int32_t* bcnt, const int32_t* slot,
                                                           const int32_t* bstart, int64_t n, Parts p, WinTpl t,
                                                           const int32_t* fresh, int32_t n_fresh) {
  if (bstart[blockIdx.x] >= n_fresh || bstart[blockIdx.x + 1] == bstart[blockIdx.x]) return;   // no slot used
  int v;
  const int32_t r = win_rank(flag, bcnt, bstart, n, n_fresh, v);
  if (v && r < n_fresh) {
    const int32_t src = fresh[r];
    const int32_t i = slot[blockIdx.x * (int64_t)kWinBlock + threadIdx.x];
    p.x[i] = t.x[src]; p.y[i] = t.y[src]; p.z[i] = t.z[src]; p.w[i] = t.w[src];
    p.ux[i] = 0.0; p.uy[i] = 0.0; p.uz[i] = 0.0;
  }
}

// With dep.rho set, a placed particle also deposits its rho (global atomics: a column's
// worth of particles), for a cycle whose push deposited rho^{n+1} already.
__global__ void __launch_bounds__(kWinBlock) k_win_inject_f32(int32_t* flag, int32_t* bcnt, const int32_t* slot,
                                                               const int32_t* bstart, int64_t n, PartsF p, WinTplF t,
                                                               const int32_t* fresh, int32_t n_fresh, GeomF g,
                                                               DepArgsF dep, const float* invV) {
  if (bstart[blockIdx.x] >= n_fresh || bstart[blockIdx.x + 1] == bstart[blockIdx.x]) return;   // no slot used
  int v;
  const int32_t r = win_rank(flag, bcnt, bstart, n, n_fresh, v);
  if (v && r < n_fresh) {
    const int32_t src = fresh[r];
    const int32_t i = slot[blockIdx.x * (int64_t)kWinBlock + threadIdx.x];
    p.iz[i] = t.iz[src]; p.fz[i] = t.fz[src]; p.ixy[i] = t.ixy[src];
    p.fx[i] = t.fx[src]; p.fy[i] = t.fy[src]; p.w[i] = t.w[src];
    p.ux[i] = 0.f; p.uy[i] = 0.f; p.uz[i] = 0.f;
    p.uxl[i] = 0.f; p.uyl[i] = 0.f; p.uzl[i] = 0.f;
    if (dep.rho) {
      const int32_t c = t.ixy[src];
      deposit_rho_global(g, dep.rho, invV, dep.q, t.iz[src], t.fz[src], (float)cell_x(c) + t.fx[src],
                         (float)cell_y(c) + t.fy[src], t.w[src]);
    }
  }
}

}  // namespace

bool is_mixed(const Sim* s) { return s->cfg.precision != PIC_FP64; }

// Kernel instances of the mixed form by mode count (1..kMaxModes).
using DepositKernel = void (*)(const PartsF, int64_t, GeomF, DepArgsF, const float*, int32_t*, BandArgs);
using GatherPushKernel = void (*)(PartsF, int64_t, GeomF, const float2* __restrict__, float, float, float, float,
                                  DepArgsF, const float*, int, int32_t*, BandArgs, WinArgs);

template <int NM>
DepositKernel deposit_kernel_nm(int kind) {
  return kind == 1 ? k_deposit_f32<NM, 1> : kind == 2 ? k_deposit_f32<NM, 2> : k_deposit_f32<NM, 3>;
}

DepositKernel deposit_kernel(int nm, int kind) {
  switch (nm) {
    case 1: return deposit_kernel_nm<1>(kind);
    case 2: return deposit_kernel_nm<2>(kind);
    case 3: return deposit_kernel_nm<3>(kind);
    default: return deposit_kernel_nm<4>(kind);
  }
}

template <int NM>
GatherPushKernel gather_push_kernel_nm(bool win, bool rho) {
  return win ? (rho ? k_gather_push_f32<NM, true, true> : k_gather_push_f32<NM, true, false>)
             : (rho ? k_gather_push_f32<NM, false, true> : k_gather_push_f32<NM, false, false>);
}

GatherPushKernel gather_push_kernel(int nm, bool win, bool rho) {
  switch (nm) {
    case 1: return gather_push_kernel_nm<1>(win, rho);
    case 2: return gather_push_kernel_nm<2>(win, rho);
    case 3: return gather_push_kernel_nm<3>(win, rho);
    default: return gather_push_kernel_nm<4>(win, rho);
  }
}

// Shared-memory bands for the deposits: chunks of cell-sorted particles per CTA (1024, or
// the tuned size: a power of two) and a
// band of ncomp components (all modes, 16 bytes per complex node) within kBandBudget, so
// that two CTAs fit on an SM: 8 or 4 full z-rows when they fit, else 4 rows of as many r
// nodes as fit (at least 16).  jmargin: r nodes a particle can move before it deposits.
constexpr size_t kBandBudget = 104 * 1024;
struct BandPlan {
  BandArgs args;
  size_t smem;
};
BandPlan band_plan(const Sim* s, int ncomp, int jmargin) {
  const pic_config& c = s->cfg;
  const int64_t chunk = s->tune_chunk > 0 ? s->tune_chunk : 1024;
  int lg = 0;
  while ((int64_t(1) << lg) < chunk) ++lg;
  BandPlan bp{BandArgs{chunk, 0, 0, jmargin, lg}, 0};
  if (ncomp <= 0) return bp;
  // one r node of one row: re hi, re lo for every mode, im hi, im lo for the modes m >= 1,
  // plus one padding word; a row is padded by up to 31 words (BandF)
  const size_t node_words = (size_t)band_node_words(c.Nm, ncomp);
  const size_t row_bytes = (node_words * c.Nr + 31) * sizeof(int32_t);
  int tz = 0, jw = 0;
  if (kBandBudget / row_bytes >= 4) {
    tz = kBandBudget / row_bytes >= 8 ? 8 : 4;   // a power of two (Nz >= 8)
    jw = c.Nr;
  } else {
    tz = 4;
    jw = std::min(c.Nr, (int)((kBandBudget / (4 * sizeof(int32_t)) - 31) / node_words));
    if (jw < 16) return bp;
  }
  bp.args.tz = tz;
  bp.args.jw_max = jw;
  bp.smem = (size_t)tz * (jw * node_words + 31) * sizeof(int32_t);
  return bp;
}

pic_status launch_sort(Sim* s) {
  const int64_t np = s->np;
  const int ncell = s->cfg.Nz * s->cfg.Nr;
  int32_t* keys = s->at<int32_t>(s->lay.keys);
  int32_t* count = s->at<int32_t>(s->lay.count);
  int32_t* start = s->at<int32_t>(s->lay.start);
  int32_t* blk = s->at<int32_t>(s->lay.scan_blk);
  int32_t* tmp = s->at<int32_t>(s->lay.perm_tmp);
  int32_t* perm = s->at<int32_t>(s->lay.perm);
  int32_t* big_list = s->at<int32_t>(s->lay.big_list);
  int32_t* big_count = s->at<int32_t>(s->lay.big_count);
  int32_t* err = s->at<int32_t>(s->lay.err);
  int32_t* cursor = reinterpret_cast<int32_t*>(s->at<char>(s->lay.scan_blk) + 4 * 4096 * sizeof(int32_t));
  int32_t* slot = s->win.on ? reinterpret_cast<int32_t*>(s->win.ws + s->win.slot) : nullptr;
  PIC_CUDA(cudaMemsetAsync(count, 0, sizeof(int32_t) * (ncell + kTailBins + 1), s->stream));   // cells + inactive
  PIC_CUDA(cudaMemsetAsync(big_count, 0, 2 * sizeof(int32_t), s->stream));
  if (np == 0) return PIC_OK;
  const bool win = slot != nullptr;
  if (is_mixed(s)) {
    if (win)
      k_keys_f32<true><<<pgrid(np), 256, 0, s->stream>>>(partsf_of(s, s->cur), np, geomf_of(s), keys, count, err);
    else
      k_keys_f32<false><<<pgrid(np), 256, 0, s->stream>>>(partsf_of(s, s->cur), np, geomf_of(s), keys, count, err);
  } else {
    if (win)
      k_keys<true><<<pgrid(np), 256, 0, s->stream>>>(parts_of(s, s->cur), np, geom_of(s), keys, count, err);
    else
      k_keys<false><<<pgrid(np), 256, 0, s->stream>>>(parts_of(s, s->cur), np, geom_of(s), keys, count, err);
  }
  PIC_LAUNCHED(s);
  const int nbin = ncell + kTailBins;
  const int nblk = (nbin + kScanBlock - 1) / kScanBlock;
  k_scan_local<<<nblk, kScanThreads, 0, s->stream>>>(count, start, blk, nbin);
  PIC_LAUNCHED(s);
  k_scan_blocks<<<1, kScanThreads, 0, s->stream>>>(blk, nblk, start, nbin);
  PIC_LAUNCHED(s);
  k_scan_add<<<pgrid(nbin), 256, 0, s->stream>>>(start, blk, nbin, cursor);
  PIC_LAUNCHED(s);
  if (win)
    k_scatter<true><<<pgrid(np), 256, 0, s->stream>>>(keys, np, cursor, tmp, ncell);
  else
    k_scatter<false><<<pgrid(np), 256, 0, s->stream>>>(keys, np, cursor, tmp, ncell);
  PIC_LAUNCHED(s);
  k_cell_sort_small<<<pgrid(ncell), 256, 0, s->stream>>>(start, tmp, perm, ncell, big_list, big_count);
  PIC_LAUNCHED(s);
  k_cell_sort_big<<<152 * 4, 256, 0, s->stream>>>(start, tmp, perm, big_list, big_count, ncell, win ? 1 : 0);
  PIC_LAUNCHED(s);
  if (is_mixed(s))
    if (win)
      k_permute_f32<true><<<pgrid(np), 256, 0, s->stream>>>(partsf_of(s, s->cur), partsf_of(s, 1 - s->cur), perm, np,
                                                            slot);
    else
      k_permute_f32<false><<<pgrid(np), 256, 0, s->stream>>>(partsf_of(s, s->cur), partsf_of(s, 1 - s->cur), perm, np,
                                                             slot);
  else if (win)
    k_permute<true><<<pgrid(np), 256, 0, s->stream>>>(parts_of(s, s->cur), parts_of(s, 1 - s->cur), perm, np, slot);
  else
    k_permute<false><<<pgrid(np), 256, 0, s->stream>>>(parts_of(s, s->cur), parts_of(s, 1 - s->cur), perm, np, slot);
  PIC_LAUNCHED(s);
  s->cur = 1 - s->cur;
  return PIC_OK;
}

// Inverse ring volumes 1/(2 pi r_j dr dz), at the tail of the diagnostics block, built once.
pic_status build_inv_volume(Sim* s) {
  double* base = s->at<double>(s->lay.diag_acc) + 64 + 3 * (size_t)kMaxSlices;
  if (is_mixed(s))
    k_inv_volume_f<<<(s->cfg.Nr + 127) / 128, 128, 0, s->stream>>>(reinterpret_cast<float*>(base), s->cfg.Nr,
                                                                    s->cfg.dr, s->cfg.dz);
  else
    k_inv_volume<<<(s->cfg.Nr + 127) / 128, 128, 0, s->stream>>>(base, s->cfg.Nr, s->cfg.dr, s->cfg.dz);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

static double* inv_volume(Sim* s) { return s->at<double>(s->lay.diag_acc) + 64 + 3 * (size_t)kMaxSlices; }

pic_status launch_deposit(Sim* s, int32_t what, int32_t id_lo, int32_t id_hi, void* rho_out) {
  const size_t G = s->grid_elems();
  int32_t* err = s->at<int32_t>(s->lay.err);
  if (is_mixed(s)) {
    DepArgsF a;
    a.q = (float)s->cfg.q;
    a.id_lo = id_lo;
    a.id_hi = id_hi;
    a.rho = (what & PIC_DEP_RHO) ? (rho_out ? (float2*)rho_out : s->at<float2>(s->lay.dep)) : nullptr;
    a.J = (what & PIC_DEP_J) ? s->at<float2>(s->lay.dep) + G : nullptr;
    if (a.J) PIC_CUDA(cudaMemsetAsync(a.J, 0, 3 * G * sizeof(float2), s->stream));
    if (s->np == 0) return PIC_OK;
    const int kind = (a.rho ? 1 : 0) | (a.J ? 2 : 0);
    if (kind == 0) return PIC_OK;
    const BandPlan bp = band_plan(s, (kind & 1 ? 1 : 0) + (kind & 2 ? 3 : 0), 1);
    auto* kern = deposit_kernel(s->cfg.Nm, kind);
    kern<<<(int)((s->np + bp.args.chunk - 1) / bp.args.chunk), kBandThreads, bp.smem, s->stream>>>(
        partsf_of(s, s->cur), s->np, geomf_of(s), a, reinterpret_cast<const float*>(inv_volume(s)), err, bp.args);
  } else {
    DepArgs a;
    a.q = s->cfg.q;
    a.id_lo = id_lo;
    a.id_hi = id_hi;
    a.rho = (what & PIC_DEP_RHO) ? (rho_out ? (double2*)rho_out : s->at<double2>(s->lay.dep)) : nullptr;
    a.J = (what & PIC_DEP_J) ? s->at<double2>(s->lay.dep) + G : nullptr;
    if (a.J) PIC_CUDA(cudaMemsetAsync(a.J, 0, 3 * G * sizeof(double2), s->stream));
    if (s->np == 0) return PIC_OK;
    k_deposit<<<pgrid(s->np), 256, 0, s->stream>>>(parts_of(s, s->cur), s->np, geom_of(s), a, inv_volume(s), err);
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_gather_push(Sim* s, int32_t fuse_current, const WinArgs& wa, bool fuse_rho, cudaEvent_t after_layout) {
  const size_t G = s->grid_elems();
  int32_t* err = s->at<int32_t>(s->lay.err);
  const pic_config& c = s->cfg;
  if (is_mixed(s)) {
    fuse_rho = fuse_rho && fuse_current;
    DepArgsF a;
    a.q = (float)c.q;
    a.id_lo = INT32_MIN;
    a.id_hi = INT32_MAX;
    a.rho = fuse_rho ? s->at<float2>(s->lay.dep) : nullptr;
    a.J = s->at<float2>(s->lay.dep) + G;
    if (s->np == 0) {
      if (fuse_current) PIC_CUDA(cudaMemsetAsync(a.J, 0, 3 * G * sizeof(float2), s->stream));
      if (fuse_rho)   // rho^{n+1} starts from the immobile background
        PIC_CUDA(cudaMemcpyAsync(a.rho, s->at<float2>(s->lay.rho_ion), G * sizeof(float2), cudaMemcpyDeviceToDevice,
                                 s->stream));
      if (after_layout) PIC_CUDA(cudaEventRecord(after_layout, s->stream));
      return PIC_OK;
    }
    const float kq = (float)(c.q * c.dt / (2.0 * c.mass * kC));
    const float kqc = (float)(c.q * c.dt / (2.0 * c.mass));
    const float chdt_dr = (float)(0.5 * kC * c.dt / c.dr);
    const float chdt_dz = (float)(0.5 * kC * c.dt / c.dz);
    // a half step moves a particle by at most c dt / 2 in r (a full step, for rho, c dt)
    const BandPlan bp = band_plan(s, fuse_current ? (fuse_rho ? 4 : 3) : 0,
                                  1 + (int)std::ceil((fuse_rho ? 1.0 : 0.5) * kC * c.dt / c.dr));
    // E and B (adjacent, 6 x Nm planes) into the node-major gather layout
    const int NV = 6 * c.Nm, tr = NV <= 12 ? 8 : 4;
    dim3 tgrid((c.Nz + 31) / 32, (c.Nr + tr - 1) / tr);
    k_nodes_rz<<<tgrid, 256, 32 * (tr * NV + 1) * sizeof(float2), s->stream>>>(
        s->at<float2>(s->lay.E), s->at<float2>(s->lay.ebt), c.Nr, c.Nz, NV, tr, a.J, fuse_current ? (int)(3 * G) : 0,
        a.rho, s->at<float2>(s->lay.rho_ion), fuse_rho ? (int)G : 0);
    PIC_LAUNCHED(s);
    if (after_layout) PIC_CUDA(cudaEventRecord(after_layout, s->stream));
    const int nblk = (int)((s->np + bp.args.chunk - 1) / bp.args.chunk);
    auto* kern = gather_push_kernel(c.Nm, wa.on != 0, fuse_rho);
    kern<<<nblk, kBandThreads, bp.smem, s->stream>>>(
        partsf_of(s, s->cur), s->np, geomf_of(s), s->at<float2>(s->lay.ebt), kq, kqc, chdt_dr, chdt_dz, a,
        reinterpret_cast<const float*>(inv_volume(s)), fuse_current, err, bp.args, wa);
  } else {
    if (after_layout) PIC_CUDA(cudaEventRecord(after_layout, s->stream));   // no separate layout
    const double kq = c.q * c.dt / (2.0 * c.mass);
    fuse_rho = fuse_rho && fuse_current && !wa.on;
    DepArgs a;
    a.q = c.q;
    a.id_lo = INT32_MIN;
    a.id_hi = INT32_MAX;
    a.rho = fuse_rho ? s->at<double2>(s->lay.dep) : nullptr;
    a.J = s->at<double2>(s->lay.dep) + G;
    if (fuse_current) PIC_CUDA(cudaMemsetAsync(a.J, 0, 3 * G * sizeof(double2), s->stream));
    if (fuse_rho)   // rho^{n+1} starts from the immobile background
      PIC_CUDA(cudaMemcpyAsync(a.rho, s->at<double2>(s->lay.rho_ion), G * sizeof(double2), cudaMemcpyDeviceToDevice,
                               s->stream));
    if (s->np == 0) return PIC_OK;
    const double2* E = s->at<double2>(s->lay.E);
    const double2* B = s->at<double2>(s->lay.B);
    const float4* ebdw = eb_dw_active(s) ? s->at<float4>(s->lay.ebdw) : nullptr;
    const Parts p = parts_of(s, s->cur);
    const GridGeom g = geom_of(s);
    const int grid = pgrid(s->np);
    if (wa.on && ebdw)
      k_gather_push<true, true><<<grid, 256, 0, s->stream>>>(p, s->np, g, E, B, ebdw, kq, c.dt, a, inv_volume(s),
                                                             fuse_current, err, wa);
    else if (wa.on)
      k_gather_push<true, false><<<grid, 256, 0, s->stream>>>(p, s->np, g, E, B, ebdw, kq, c.dt, a, inv_volume(s),
                                                              fuse_current, err, wa);
    else if (ebdw)
      k_gather_push<false, true><<<grid, 256, 0, s->stream>>>(p, s->np, g, E, B, ebdw, kq, c.dt, a, inv_volume(s),
                                                              fuse_current, err, wa);
    else
      k_gather_push<false, false><<<grid, 256, 0, s->stream>>>(p, s->np, g, E, B, ebdw, kq, c.dt, a,
                                                               inv_volume(s), fuse_current, err, wa);
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_diag(Sim* s, int32_t lo, int32_t hi, pic_diag* out, double* slice_sigma, int32_t max_slices) {
  const int col0 = s->win.on ? (int)(s->win.shifts % s->cfg.Nz) : 0;
  if (is_mixed(s)) {
    Acc32 a{partsf_of(s, s->cur), s->cfg.dz, s->cfg.dr, col0, s->cfg.Nz};
    return run_diag(s, a, lo, hi, out, slice_sigma, max_slices);
  }
  Acc64 a{parts_of(s, s->cur), col0 * s->cfg.dz, s->cfg.Nz * s->cfg.dz};
  return run_diag(s, a, lo, hi, out, slice_sigma, max_slices);
}

// Mixed form: float64 SoA (the staging area, or src with its stride) -> FP32 particles of
// the current buffer.
pic_status launch_particles_in(Sim* s, const int32_t* id_dev, int64_t n, const double* src, int64_t stride) {
  if (n == 0) return PIC_OK;
  if (!src) {
    src = s->at<double>(s->lay.stage64);
    stride = s->cfg.np_capacity;
  }
  k_p64_to_p32<<<pgrid(n), 256, 0, s->stream>>>(src, stride, id_dev, partsf_of(s, s->cur), n, s->cfg.Nz,
                                                 1.0 / s->cfg.dz, 1.0 / s->cfg.dr);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

// Mixed form: FP32 particles -> float64 SoA in the staging area (ids to id_dev if given).
pic_status launch_particles_out(Sim* s, int32_t* id_dev, int64_t n) {
  if (n == 0) return PIC_OK;
  k_p32_to_p64<<<pgrid(n), 256, 0, s->stream>>>(partsf_of(s, s->cur), n, s->at<double>(s->lay.stage64),
                                                 s->cfg.np_capacity, id_dev, s->cfg.dz, s->cfg.dr);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

size_t diag_acc_doubles() { return 64 + 3 * (size_t)kMaxSlices + kMaxNr + kDiagPartsDoubles; }

// The band kernels may use up to kBandBudget bytes of dynamic shared memory; the limit is
// raised once per device (a per-launch change would race between host threads).
pic_status particles_configure_device() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PIC_OK;
  for (int nm = 1; nm <= kMaxModes; ++nm) {
    for (int kind = 1; kind <= 3; ++kind)
      PIC_CUDA(cudaFuncSetAttribute(deposit_kernel(nm, kind), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kBandBudget));
    for (int v = 0; v < 4; ++v)
      PIC_CUDA(cudaFuncSetAttribute(gather_push_kernel(nm, v & 1, v & 2), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)kBandBudget));
  }
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

// ---- moving window: particle side
size_t window_layout(const Sim* s, int64_t n_tpl, WindowState* w) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const pic_config& c = s->cfg;
  const size_t cap = (size_t)std::max<int64_t>(c.np_capacity, 1);
  const size_t rows = 6 * (size_t)c.Nm * c.Nr;
  WindowState t;
  t.tpl = take(32 * (size_t)std::max<int64_t>(n_tpl, 1));
  t.colids = take(4 * (size_t)std::max<int64_t>(n_tpl, 1));
  t.flag = take(4 * cap);
  t.slot = take(4 * cap);
  t.bcnt = take(4 * (cap / kWinBlock + 2));
  t.bstart = take(4 * (cap / kWinBlock + 2));
  t.dropped = take(8);
  t.colv = take(16 * rows);
  t.hv = take(16 * rows);
  t.ph = take(16 * (size_t)c.Nz);
  t.hvf = take(8 * rows);
  t.phf = take(8 * (size_t)c.Nz);
  if (w) {
    w->tpl = t.tpl; w->colids = t.colids; w->flag = t.flag; w->slot = t.slot; w->bcnt = t.bcnt;
    w->bstart = t.bstart;
    w->dropped = t.dropped; w->colv = t.colv; w->hv = t.hv; w->ph = t.ph; w->hvf = t.hvf; w->phf = t.phf;
  }
  return off;
}

pic_status launch_window_reserve(Sim* s, int64_t n_reserve) {
  if (n_reserve <= 0) return PIC_OK;
  const int64_t first = s->np;
  if (is_mixed(s))
    k_win_reserve_f32<<<pgrid(n_reserve), 256, 0, s->stream>>>(partsf_of(s, s->cur), first, n_reserve,
                                                                (int32_t)first, s->cfg.Nz, s->cfg.Nr);
  else
    k_win_reserve<<<pgrid(n_reserve), 256, 0, s->stream>>>(parts_of(s, s->cur), first, n_reserve, (int32_t)first,
                                                            s->cfg.Nz, s->cfg.Nr, s->cfg.dz, s->cfg.dr);
  PIC_LAUNCHED(s);
  s->np += n_reserve;
  return PIC_OK;
}

pic_status window_take_template(Sim* s, int32_t* keys_host) {
  const int64_t n = s->win.n_tpl;
  if (n == 0 || s->np == 0) return PIC_OK;
  int32_t* col = s->at<int32_t>(s->lay.perm_tmp);   // scratch, capacity >= n
  if (is_mixed(s))
    k_win_template_f32<<<pgrid(s->np), 256, 0, s->stream>>>(partsf_of(s, s->cur), s->np, n, win_tplf(s), col);
  else
    k_win_template<<<pgrid(s->np), 256, 0, s->stream>>>(parts_of(s, s->cur), s->np, n, win_tpl(s), col, s->cfg.Nz,
                                                         s->cfg.dz);
  PIC_LAUNCHED(s);
  PIC_CUDA(cudaMemcpyAsync(keys_host, col, n * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
  PIC_CUDA(cudaStreamSynchronize(s->stream));
  return PIC_OK;
}

pic_status launch_window_mark_all(Sim* s) {
  WindowState& w = s->win;
  int32_t* flag = reinterpret_cast<int32_t*>(w.ws + w.flag);
  int32_t* slot = reinterpret_cast<int32_t*>(w.ws + w.slot);
  int32_t* bcnt = reinterpret_cast<int32_t*>(w.ws + w.bcnt);
  if (s->np == 0) return PIC_OK;
  if (is_mixed(s)) {
    const PartsF p = partsf_of(s, s->cur);
    k_win_mark_all<float><<<pgrid(s->np), 256, 0, s->stream>>>(p.w, p.id, s->np, flag, slot, bcnt);
  } else {
    const Parts p = parts_of(s, s->cur);
    k_win_mark_all<double><<<pgrid(s->np), 256, 0, s->stream>>>(p.w, p.id, s->np, flag, slot, bcnt);
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_window_inject(Sim* s, int column, bool deposit_rho) {
  WindowState& w = s->win;
  const int32_t c0 = w.col_start_host[column], n_fresh = w.col_start_host[column + 1] - c0;
  int32_t* flag = reinterpret_cast<int32_t*>(w.ws + w.flag);
  const int32_t* slot = reinterpret_cast<const int32_t*>(w.ws + w.slot);
  int32_t* bcnt = reinterpret_cast<int32_t*>(w.ws + w.bcnt);
  int32_t* bstart = reinterpret_cast<int32_t*>(w.ws + w.bstart);
  const int32_t* fresh = reinterpret_cast<const int32_t*>(w.ws + w.colids) + c0;
  auto* dropped = reinterpret_cast<unsigned long long*>(w.ws + w.dropped);
  const int nb = (int)((w.n_ids + kWinBlock - 1) / kWinBlock);
  if (nb == 0) return PIC_OK;
  k_win_bscan<<<1, kWinBlock, 0, s->stream>>>(bcnt, bstart, nb, n_fresh, dropped);
  PIC_LAUNCHED(s);
  if (n_fresh == 0) return PIC_OK;
  if (is_mixed(s)) {
    DepArgsF a;
    a.q = (float)s->cfg.q;
    a.id_lo = INT32_MIN;
    a.id_hi = INT32_MAX;
    a.rho = deposit_rho ? s->at<float2>(s->lay.dep) : nullptr;
    a.J = nullptr;
    k_win_inject_f32<<<nb, kWinBlock, 0, s->stream>>>(flag, bcnt, slot, bstart, w.n_ids, partsf_of(s, s->cur),
                                                       win_tplf(s), fresh, n_fresh, geomf_of(s), a,
                                                       reinterpret_cast<const float*>(inv_volume(s)));
  }
  else
    k_win_inject<<<nb, kWinBlock, 0, s->stream>>>(flag, bcnt, slot, bstart, w.n_ids, parts_of(s, s->cur), win_tpl(s),
                                                   fresh, n_fresh);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
