// Batched complex DFT along z (a5, a9): Fourier transform along z of the
// quasi-cylindrical scheme (section "Finite order pseudo-spectral solvers").
//   forward: Fhat(k) = sum_i F(z_i) e^{-2 pi i k i / Nz}
//   inverse: F(z_i) = (1/Nz) sum_k Fhat(k) e^{+2 pi i k i / Nz}
// Power-of-two lengths use radix-8 passes with the values in registers (k_fft_pow2 for
// double rows; k_fft_pow2_tma for float rows, persistent and fed by bulk copies); other
// 7-smooth lengths a mixed-radix (8, 4, 2, 3, 5, 7) self-sorting Stockham sequence of passes
// between two shared row buffers (k_fft_rows).  All read per-pass twiddle tables.  Any
// other length goes through Bluestein's chirp-z algorithm on power-of-two rows (below).
// The component combination of the quasi-cylindrical scheme is fused into the row load:
// out = ca * inA + cb * inB, which forms J_+- = (J_r -+ i J_theta)/2 before the forward
// transform and E_r = E_+ + E_-, E_theta = i (E_+ - E_-) before the inverse one.
#include <mutex>
#include <type_traits>

#include "pic_internal.cuh"
#include "dword.cuh"
#include "tc_common.cuh"

namespace pic {
namespace {

template <typename R> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };

template <> struct Vec2<dw> { using T = dw2; };

template <typename T> __device__ __forceinline__ T cmul(T a, T b) {
  T r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T> __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename T> __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
// multiply by -i (forward) or +i (inverse)
template <typename T, bool INV> __device__ __forceinline__ T mul_mi(T a) {
  T r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}

// v with its sign flipped when neg, by integer operations (no float64 instruction).
__device__ __forceinline__ double neg_if(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ (neg ? (long long)0x8000000000000000ULL : 0LL));
}
__device__ __forceinline__ float neg_if(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ (neg ? (int)0x80000000u : 0));
}

// c x for a combination coefficient c of kind 0 (real), 1 (imaginary) or 2 (general); in
// double rows a coefficient +-1 or +-i (unit != 0) costs sign flips only and a real or
// imaginary one two multiplies (those rows are bound by the float64 unit).  Float rows
// multiply in full: branches there would keep the row loads from issuing together.
template <typename T>
__device__ __forceinline__ T coef_mul(T c, int kind, int unit, T x) {
  if constexpr (sizeof(x.x) == 4) return cmul(c, x);
  T r;
  if (kind == 0) {
    if (unit) { r.x = neg_if(x.x, unit < 0); r.y = neg_if(x.y, unit < 0); }
    else { r.x = c.x * x.x; r.y = c.x * x.y; }
  } else if (kind == 1) {   // i c.y x = (-c.y x.y, c.y x.x)
    if (unit) { r.x = neg_if(x.y, unit > 0); r.y = neg_if(x.x, unit < 0); }
    else { r.x = -c.y * x.y; r.y = c.y * x.x; }
  } else {
    r = cmul(c, x);
  }
  return r;
}

// The combination coefficients of component comp for rows of type R.
template <typename R, typename C2>
__device__ __forceinline__ void row_coefs(const RowCombine& rc, int comp, C2& ca, C2& cb, int& ka, int& kb, int& ua,
                                          int& ub) {
  if constexpr (sizeof(R) == 4) {
    ca.x = rc.fcaRe[comp]; ca.y = rc.fcaIm[comp];
    cb.x = rc.fcbRe[comp]; cb.y = rc.fcbIm[comp];
  } else if constexpr (std::is_same<R, dw>::value) {   // the coefficients are exact in float
    ca.x = dw(rc.fcaRe[comp], 0.f); ca.y = dw(rc.fcaIm[comp], 0.f);
    cb.x = dw(rc.fcbRe[comp], 0.f); cb.y = dw(rc.fcbIm[comp], 0.f);
  } else {
    ca.x = rc.caRe[comp]; ca.y = rc.caIm[comp];
    cb.x = rc.cbRe[comp]; cb.y = rc.cbIm[comp];
  }
  ka = rc.kindA[comp]; kb = rc.kindB[comp];
  ua = rc.unitA[comp]; ub = rc.unitB[comp];
}

// 1/sqrt(2) and 1/N in the row arithmetic R.
template <typename R> __device__ __forceinline__ R inv_sqrt2() { return (R)0.70710678118654752440; }
template <> __device__ __forceinline__ dw inv_sqrt2<dw>() { return dw(0.70710676908493042f, 1.2101617485882343e-08f); }
template <typename R> __device__ __forceinline__ R inv_len(int N) { return (R)1 / (R)N; }
template <> __device__ __forceinline__ dw inv_len<dw>(int N) { return dw(1.f / (float)N, 0.f); }   // N a power of two


// Element type of the rows in global memory for row arithmetic R (double-word rows are
// stored as doubles), and the conversions between the two.
template <typename R> struct GlobalOf { using T = typename Vec2<R>::T; };
template <> struct GlobalOf<dw> { using T = double2; };
template <typename C2, typename G2> __device__ __forceinline__ C2 from_global(const G2& v) {
  if constexpr (std::is_same<C2, G2>::value) {
    return v;
  } else {
    C2 r;
    r.x = dw_from_double(v.x);
    r.y = dw_from_double(v.y);
    return r;
  }
}
__device__ __forceinline__ double2 to_global(const dw2& v) { return make_double2(dw_to_double(v.x), dw_to_double(v.y)); }
__device__ __forceinline__ float2 to_global(const float2& v) { return v; }
__device__ __forceinline__ double2 to_global(const double2& v) { return v; }

struct FftPlan {
  int N;
  int n_pass;
  int radix[kMaxRadixPasses];
};

// ---- power-of-two rows ----
// Self-sorting Stockham passes of radix 8 (then one radix-2 or radix-4 pass when log2 N is
// not a multiple of 3).  Pass p (radix R, L = product of the earlier radices) maps
//   y_s = sum_r v_r w_R^{rs},  v_r = x[t + r N/R] w_{LR}^{r k},  k = t mod L, j = t / L,
//   out[j L R + s L + k] = y_s,
// so the first pass reads a row in natural order and the last pass (L = N/R, j = 0)
// writes it in natural order: both go straight between global memory and registers.
// Each thread holds E values of its row; the intermediate passes exchange them through one
// row buffer in shared memory, padded by one element per 128 bytes against bank conflicts.
// The twiddles w_{LR}^{rk} of pass (R, L) sit at table entry L-1 + (r-1) L + k (the
// tables of all passes tile entries 0..N-2), so a warp reads consecutive entries.
constexpr int kFftThreads = 256;

// Resident CTAs per SM asked of the register allocator for E values per thread (double rows
// and the Bluestein rows).  Float rows of 4096 and 8192 points (E = 16, 32) trade a few
// spilled bytes for 3 and 2 CTAs per SM: with one CTA per SM a row's loads, passes and
// stores ran one after another on the SM.
template <typename R> constexpr int fft_min_ctas(int E) {
  return E == 8 ? 4 : (E == 16 ? (sizeof(R) == 4 ? 3 : 2) : (sizeof(R) == 4 ? 2 : 1));
}

template <typename C2, bool INV> __device__ __forceinline__ C2 conj_if(C2 w) {
  if (INV) w.y = -w.y;
  return w;
}

template <typename C2, bool INV> __device__ __forceinline__ void dft2(C2* v) {
  const C2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <typename C2, bool INV> __device__ __forceinline__ void dft4(C2* v) {
  const C2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
  const C2 s13 = cadd(v[1], v[3]), d13 = mul_mi<C2, INV>(csub(v[1], v[3]));
  v[0] = cadd(s02, s13);
  v[1] = cadd(d02, d13);
  v[2] = csub(s02, s13);
  v[3] = csub(d02, d13);
}

// 8-point DFT as two 4-point DFTs: even outputs from a_r = v_r + v_{r+4}, odd outputs from
// b_r = (v_r - v_{r+4}) w_8^r.
template <typename C2, bool INV> __device__ __forceinline__ void dft8(C2* v) {
  using R = decltype(v[0].x);
  const R h = inv_sqrt2<R>();
  C2 a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = csub(v[r], v[r + 4]);
  }
  {   // w_8^1 = (1 -+ i)/sqrt(2)
    const C2 x = b[1];
    if (INV) { b[1].x = h * (x.x - x.y); b[1].y = h * (x.x + x.y); }
    else     { b[1].x = h * (x.x + x.y); b[1].y = h * (x.y - x.x); }
  }
  b[2] = mul_mi<C2, INV>(b[2]);   // w_8^2 = -+ i
  {   // w_8^3 = (-1 -+ i)/sqrt(2)
    const C2 x = b[3];
    if (INV) { b[3].x = -h * (x.x + x.y); b[3].y = h * (x.x - x.y); }
    else     { b[3].x = h * (x.y - x.x); b[3].y = -h * (x.x + x.y); }
  }
  dft4<C2, INV>(a);
  dft4<C2, INV>(b);
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    v[2 * r] = a[r];
    v[2 * r + 1] = b[r];
  }
}

// Per-row context of the power-of-two kernel.
template <typename C2, typename G2 = C2> struct RowCtx {
  const G2* a;    // source rows of the combination (b may be null), in global memory
  const G2* b;
  C2 ca, cb;
  int ka, kb, ua, ub;   // coefficient kinds and units (coef_mul)
  G2* o;          // destination row
  float4* odw;    // double-word copy of the destination row (double-word rows only; may be null)
  C2* buf;        // padded shared row buffer
  int N, tr, TR;
  bool active;    // false for the idle row slots of the last CTA
};

template <int PS> __device__ __forceinline__ int padded(int i) { return i + (i >> PS); }

// Inputs of the first pass (radix 8): v[8q + r] = (ca a + cb b)[t + r N/8], t = tr + q TR.
template <typename C2, int E, typename G2>
__device__ __forceinline__ void pow2_load_global(C2 (&v)[E], const RowCtx<C2, G2>& c) {
  using Re = decltype(v[0].x);
  const int N8 = c.N >> 3;
#pragma unroll
  for (int q = 0; q < E / 8; ++q) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = c.tr + q * c.TR + r * N8;
      C2 x;
      x.x = (Re)0; x.y = (Re)0;
      if (c.active) {
        x = coef_mul(c.ca, c.ka, c.ua, from_global<C2>(c.a[idx]));
        if (c.b) x = cadd(x, coef_mul(c.cb, c.kb, c.ub, from_global<C2>(c.b[idx])));
      }
      v[q * 8 + r] = x;
    }
  }
}

// Inputs of a later pass of radix R from the shared row buffer.
template <typename C2, int E, int R, int PS, typename G2>
__device__ __forceinline__ void pow2_load_shared(C2 (&v)[E], const RowCtx<C2, G2>& c) {
  const int NR = c.N / R;
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
#pragma unroll
    for (int r = 0; r < R; ++r) v[q * R + r] = c.buf[padded<PS>(c.tr + q * c.TR + r * NR)];
  }
}

// Twiddles w^r = w_{LR}^{rk}, r = 1 .. R-1, of butterfly k of pass (R, L).  Float rows read
// w^1 from the table and form the other powers with at most three products each (w^2 = w w,
// w^3 = w^2 w, w^4 = w^2 w^2, w^5 = w^4 w, w^6 = w^4 w^2, w^7 = w^4 w^3), a few float
// roundings from the tabulated values: one table read per butterfly instead of R - 1, which
// the register budget of 16 and 32 values per thread could not keep in flight.  Double rows
// read every power: their products would run on the float64 unit, which bounds those rows.
template <typename C2, int R>
__device__ __forceinline__ void pass_twiddles(C2 (&w)[R], const C2* __restrict__ twp, int L, int k) {
  using Re = decltype(w[0].x);
  if constexpr (sizeof(Re) == 4) {
    w[1] = twp[L - 1 + k];
    if constexpr (R > 2) {
      w[2] = cmul(w[1], w[1]);
      w[3] = cmul(w[2], w[1]);
    }
    if constexpr (R > 4) {
      w[4] = cmul(w[2], w[2]);
      w[5] = cmul(w[4], w[1]);
      w[6] = cmul(w[4], w[2]);
      w[7] = cmul(w[4], w[3]);
    }
  } else {
#pragma unroll
    for (int r = 1; r < R; ++r) w[r] = twp[L - 1 + (r - 1) * L + k];
  }
}

// Twiddles and the R-point DFTs of a pass.
template <typename C2, bool INV, int E, int R, typename G2>
__device__ __forceinline__ void pow2_butterflies(C2 (&v)[E], const RowCtx<C2, G2>& c, const C2* __restrict__ twp,
                                                 int L) {
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    if (L > 1) {
      const int k = (c.tr + q * c.TR) & (L - 1);
      C2 w[R];
      pass_twiddles<C2, R>(w, twp, L, k);
#pragma unroll
      for (int r = 1; r < R; ++r) v[q * R + r] = cmul(v[q * R + r], conj_if<C2, INV>(w[r]));
    }
    if (R == 8) dft8<C2, INV>(&v[q * R]);
    else if (R == 4) dft4<C2, INV>(&v[q * R]);
    else dft2<C2, INV>(&v[q * R]);
  }
}

// Outputs of a pass: out[j L R + s L + k] = y_s, to the shared buffer or (last pass, L =
// N/R) to the destination row, scaled by 1/N for the inverse transform.
template <typename C2, bool INV, int E, int R, int PS, typename G2>
__device__ __forceinline__ void pow2_store(C2 (&v)[E], const RowCtx<C2, G2>& c, int L, int lgL, bool last) {
  using Re = decltype(v[0].x);
  const Re scale = INV ? inv_len<Re>(c.N) : (Re)1;
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int t = c.tr + q * c.TR;
    const int base = ((t >> lgL) * R) * L + (t & (L - 1));
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) {
      const int idx = base + s2 * L;
      if (last) {
        if (c.active) {
          C2 y = v[q * R + s2];
          if (INV) {
            y.x = y.x * scale;
            y.y = y.y * scale;
          }
          c.o[idx] = to_global(y);
          if constexpr (std::is_same<C2, dw2>::value) {
            if (c.odw) c.odw[idx] = make_float4(y.x.hi, y.x.lo, y.y.hi, y.y.lo);
          }
        }
      } else {
        c.buf[padded<PS>(idx)] = v[q * R + s2];
      }
    }
  }
}

template <typename C2, bool INV, int E, int R, int PS, typename G2>
__device__ __forceinline__ void pow2_pass(C2 (&v)[E], const RowCtx<C2, G2>& c, const C2* __restrict__ twp, int L,
                                          int lgL, bool last) {
  pow2_butterflies<C2, INV, E, R>(v, c, twp, L);
  pow2_store<C2, INV, E, R, PS>(v, c, L, lgL, last);
}

// Double rows: one CTA of 256 threads transforms 256 E / N rows (N <= 2048: E = 8; N = 4096,
// 8192: one row with E = 16, 32).  Float rows take k_fft_pow2_tma below.
template <typename R, bool INV, int E>
__global__ void __launch_bounds__(kFftThreads, fft_min_ctas<R>(E)) k_fft_pow2(const typename GlobalOf<R>::T* __restrict__ in,
                                                          typename GlobalOf<R>::T* __restrict__ out,
                                                          const typename Vec2<R>::T* __restrict__ twp,
                                                          RowCombine rc, int N, int lgN, int rows,
                                                          int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  using G2 = typename GlobalOf<R>::T;
  constexpr int PS = sizeof(R) == 4 ? 4 : 3;   // one pad element per 128 bytes
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowCtx<C2, G2> c;
  c.N = N;
  c.TR = N / E;
  const int lr = threadIdx.x / c.TR;
  c.tr = threadIdx.x - lr * c.TR;
  const int row = blockIdx.x * (kFftThreads / c.TR) + lr;
  c.active = row < rows;
  c.buf = reinterpret_cast<C2*>(smem_raw) + (size_t)lr * (N + (N >> PS));
  const int rrow = c.active ? row : 0;
  const int comp = rrow / rows_per_comp;
  const int rr = rrow - comp * rows_per_comp;
  c.a = in + ((size_t)rc.srcA[comp] * rows_per_comp + rr) * N;
  const int sb = rc.srcB[comp];
  c.b = sb >= 0 ? in + ((size_t)sb * rows_per_comp + rr) * N : nullptr;
  row_coefs<R>(rc, comp, c.ca, c.cb, c.ka, c.kb, c.ua, c.ub);
  c.o = out + (size_t)rrow * N;
  c.odw = nullptr;
  if constexpr (std::is_same<C2, dw2>::value) {
    if (rc.out_dw) c.odw = reinterpret_cast<float4*>(rc.out_dw) + (size_t)rrow * N;
  }
  C2 v[E];
  const int n8 = lgN / 3, rem = lgN - 3 * n8;   // n8 >= 1 radix-8 passes, then radix 2^rem
  pow2_load_global<C2, E>(v, c);
  int L = 1, lgL = 0;
  for (int p = 0; p < n8; ++p) {
    const bool last = p == n8 - 1 && rem == 0;
    pow2_pass<C2, INV, E, 8, PS>(v, c, twp, L, lgL, last);
    if (last) return;
    L <<= 3;
    lgL += 3;
    __syncthreads();   // the pass's outputs are in the buffer
    if (p + 1 < n8) pow2_load_shared<C2, E, 8, PS>(v, c);
    else if (rem == 2) pow2_load_shared<C2, E, 4, PS>(v, c);
    else pow2_load_shared<C2, E, 2, PS>(v, c);
    __syncthreads();   // the buffer is read in full before it is rewritten
  }
  if (rem == 2) pow2_pass<C2, INV, E, 4, PS>(v, c, twp, L, lgL, true);
  else pow2_pass<C2, INV, E, 2, PS>(v, c, twp, L, lgL, true);
}

// ---- power-of-two float rows: persistent CTAs fed by bulk copies ----
// (3 x 1024 x 8192 rows, forward: 1.14 ms with k_fft_pow2 at 2 CTAs per SM, 1.89 ms at
// one, 0.66 ms here.)
// One CTA of 512 threads per SM (two for E = 8) walks groups of G = 512 E / N rows of one
// component (groups do not cross components, so each source is one contiguous run of G
// rows).  A group's source rows arrive in a shared staging area by one bulk copy per source
// (cp.async.bulk, completion counted on an mbarrier); as soon as every thread holds its
// first-pass inputs in registers, thread 0 starts the copy of the CTA's next group, which
// then runs under the passes and stores of this one.  The passes are those of k_fft_pow2
// (the first reads the combination from the staging area, the last writes the row to
// global memory).  The float rows are bound by memory latency otherwise: a CTA that loads
// its row itself waits for it before every row.
constexpr int kFftTmaThreads = 512;

template <int E> constexpr int fft_tma_ctas() { return E == 8 ? 2 : 1; }

// Float rows: E = 16 values per thread for N >= 4096, else 8; G = 512 E / N rows per group.
inline int fft_tma_e(int N) { return N >= 4096 ? 16 : 8; }
inline size_t fft_tma_smem(int N) {
  const int G = kFftTmaThreads * fft_tma_e(N) / N;
  return ((size_t)2 * G * N + (size_t)G * (N + (N >> 4))) * sizeof(float2) + 16;
}

template <bool INV, int E>
__global__ void __launch_bounds__(kFftTmaThreads, fft_tma_ctas<E>())
    k_fft_pow2_tma(const float2* __restrict__ in, float2* __restrict__ out, const float2* __restrict__ twp,
                   RowCombine rc, int N, int lgN, int rows_per_comp, int n_comp, int G, int32_t* err) {
  using C2 = float2;
  constexpr int PS = 4;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int padN = N + (N >> PS);
  C2* stage_a = reinterpret_cast<C2*>(smem_raw);
  C2* stage_b = stage_a + (size_t)G * N;
  C2* cbuf = stage_b + (size_t)G * N;
  uint64_t* bar = reinterpret_cast<uint64_t*>(cbuf + (size_t)G * padN);
  const int gpc = (rows_per_comp + G - 1) / G;   // groups per component
  const int n_groups = gpc * n_comp;
  RowCtx<C2> c;
  c.N = N;
  c.TR = N / E;
  const int lr = threadIdx.x / c.TR;              // row of the group
  c.tr = threadIdx.x - lr * c.TR;
  c.buf = cbuf + (size_t)lr * padN;
  const int n8 = lgN / 3, rem = lgN - 3 * n8;

  auto issue = [&](int g) {                      // thread 0: the copies of group g
    const int comp = g / gpc, r0 = (g - comp * gpc) * G;
    const uint32_t bytes = (uint32_t)(min(G, rows_per_comp - r0) * N * (int)sizeof(C2));
    const int sb = rc.srcB[comp];
    mbar_arrive_expect_tx(bar, sb >= 0 ? 2 * bytes : bytes);
    bulk_g2s(stage_a, in + ((size_t)rc.srcA[comp] * rows_per_comp + r0) * N, bytes, bar);
    if (sb >= 0) bulk_g2s(stage_b, in + ((size_t)sb * rows_per_comp + r0) * N, bytes, bar);
  };

  if (threadIdx.x == 0) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0 && (int)blockIdx.x < n_groups) issue(blockIdx.x);
  uint32_t parity = 0;
  for (int g = blockIdx.x; g < n_groups; g += gridDim.x, parity ^= 1u) {
    const int comp = g / gpc, r0 = (g - comp * gpc) * G;
    const int rr = r0 + lr;
    c.active = rr < rows_per_comp;
    c.a = stage_a + (size_t)lr * N;
    c.b = rc.srcB[comp] >= 0 ? stage_b + (size_t)lr * N : nullptr;
    row_coefs<float>(rc, comp, c.ca, c.cb, c.ka, c.kb, c.ua, c.ub);
    c.o = out + ((size_t)comp * rows_per_comp + (c.active ? rr : 0)) * N;
    const bool ok = mbar_wait(bar, parity);
    if (__syncthreads_or(!ok)) {                 // the copy did not complete: give up
      if (threadIdx.x == 0) {
        atomicOr(err, kErrTimeout);
        mbar_wait(bar, parity);                  // bounded: let a late copy land first
      }
      return;
    }
    C2 v[E];
    pow2_load_global<C2, E>(v, c);
    __syncthreads();                             // staging read in full
    if (threadIdx.x == 0 && g + (int)gridDim.x < n_groups) issue(g + gridDim.x);
    int L = 1, lgL = 0;
    bool done = false;
    for (int p = 0; p < n8; ++p) {
      const bool last = p == n8 - 1 && rem == 0;
      pow2_pass<C2, INV, E, 8, PS>(v, c, twp, L, lgL, last);
      if (last) { done = true; break; }
      L <<= 3;
      lgL += 3;
      __syncthreads();   // the pass's outputs are in the buffer
      if (p + 1 < n8) pow2_load_shared<C2, E, 8, PS>(v, c);
      else if (rem == 2) pow2_load_shared<C2, E, 4, PS>(v, c);
      else pow2_load_shared<C2, E, 2, PS>(v, c);
      __syncthreads();   // the buffer is read in full before it is rewritten
    }
    if (!done) {
      if (rem == 2) pow2_pass<C2, INV, E, 4, PS>(v, c, twp, L, lgL, true);
      else pow2_pass<C2, INV, E, 2, PS>(v, c, twp, L, lgL, true);
    }
  }
}

// ---- Bluestein rows in one kernel (see the chirp-z section below for the algorithm) ----
// The row of power-of-two length M stays on chip: load the N inputs times the chirp (zero
// beyond N), forward radix-8 passes ending in the shared buffer, multiply by the filter
// spectrum there, inverse passes, and store the first N outputs times the chirp.  Global
// traffic is one read and one write of the N-point rows, as for a direct transform.
template <typename C2, int E>
__device__ __forceinline__ void blue_load_global(C2 (&v)[E], const RowCtx<C2>& c, const C2* __restrict__ chirp,
                                                 int N, bool conj_chirp) {
  using Re = decltype(v[0].x);
  const int M8 = c.N >> 3;
#pragma unroll
  for (int q = 0; q < E / 8; ++q) {
#pragma unroll
    for (int r = 0; r < 8; ++r) {
      const int idx = c.tr + q * c.TR + r * M8;
      C2 x;
      x.x = (Re)0; x.y = (Re)0;
      if (c.active && idx < N) {
        x = coef_mul(c.ca, c.ka, c.ua, c.a[idx]);
        if (c.b) x = cadd(x, coef_mul(c.cb, c.kb, c.ub, c.b[idx]));
        C2 w = chirp[idx];
        if (conj_chirp) w.y = -w.y;
        x = cmul(x, w);
      }
      v[q * 8 + r] = x;
    }
  }
}

// Last inverse pass: outputs idx < N, times post(idx) = 1/M (the inverse FFT_M) times the
// outer transform's chirp factor (forward: conj(w); inverse: w / N).
template <typename C2, bool OUTER_INV, int E, int R>
__device__ __forceinline__ void blue_store_global(C2 (&v)[E], const RowCtx<C2>& c, int L, int lgL,
                                                  const C2* __restrict__ chirp, int N) {
  using Re = decltype(v[0].x);
  const Re scale = (Re)1 / (Re)c.N / (OUTER_INV ? (Re)N : (Re)1);
#pragma unroll
  for (int q = 0; q < E / R; ++q) {
    const int t = c.tr + q * c.TR;
    const int base = ((t >> lgL) * R) * L + (t & (L - 1));
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) {
      const int idx = base + s2 * L;
      if (c.active && idx < N) {
        C2 w = chirp[idx];
        if (!OUTER_INV) w.y = -w.y;
        w.x *= scale;
        w.y *= scale;
        c.o[idx] = cmul(v[q * R + s2], w);
      }
    }
  }
}

template <typename R, bool OUTER_INV, int E>
__global__ void __launch_bounds__(kFftThreads, fft_min_ctas<R>(E)) k_fft_blue(
    const typename Vec2<R>::T* __restrict__ in, typename Vec2<R>::T* __restrict__ out,
    const typename Vec2<R>::T* __restrict__ twm, const typename Vec2<R>::T* __restrict__ chirp,
    const typename Vec2<R>::T* __restrict__ spec, RowCombine rc, int N, int M, int lgM, int rows, int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  constexpr int PS = sizeof(R) == 4 ? 4 : 3;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowCtx<C2> c;
  c.N = M;
  c.TR = M / E;
  const int lr = threadIdx.x / c.TR;
  c.tr = threadIdx.x - lr * c.TR;
  const int row = blockIdx.x * (kFftThreads / c.TR) + lr;
  c.active = row < rows;
  c.buf = reinterpret_cast<C2*>(smem_raw) + (size_t)lr * (M + (M >> PS));
  const int rrow = c.active ? row : 0;
  const int comp = rrow / rows_per_comp;
  const int rr = rrow - comp * rows_per_comp;
  c.a = in + ((size_t)rc.srcA[comp] * rows_per_comp + rr) * N;
  const int sb = rc.srcB[comp];
  c.b = sb >= 0 ? in + ((size_t)sb * rows_per_comp + rr) * N : nullptr;
  row_coefs<R>(rc, comp, c.ca, c.cb, c.ka, c.kb, c.ua, c.ub);
  c.o = out + (size_t)rrow * N;
  c.odw = nullptr;
  if constexpr (std::is_same<C2, dw2>::value) {
    if (rc.out_dw) c.odw = reinterpret_cast<float4*>(rc.out_dw) + (size_t)rrow * N;
  }
  C2 v[E];
  const int n8 = lgM / 3, rem = lgM - 3 * n8;
  // forward FFT_M of the chirped, zero-padded row; every pass ends in the shared buffer
  blue_load_global<C2, E>(v, c, chirp, N, !OUTER_INV);
  int L = 1, lgL = 0;
  for (int p = 0; p < n8; ++p) {
    pow2_butterflies<C2, false, E, 8>(v, c, twm, L);
    pow2_store<C2, false, E, 8, PS>(v, c, L, lgL, false);
    L <<= 3;
    lgL += 3;
    __syncthreads();
    if (p + 1 < n8) {
      pow2_load_shared<C2, E, 8, PS>(v, c);
      __syncthreads();
    }
  }
  if (rem) {
    if (rem == 2) pow2_load_shared<C2, E, 4, PS>(v, c);
    else pow2_load_shared<C2, E, 2, PS>(v, c);
    __syncthreads();
    if (rem == 2) {
      pow2_butterflies<C2, false, E, 4>(v, c, twm, L);
      pow2_store<C2, false, E, 4, PS>(v, c, L, lgL, false);
    } else {
      pow2_butterflies<C2, false, E, 2>(v, c, twm, L);
      pow2_store<C2, false, E, 2, PS>(v, c, L, lgL, false);
    }
    __syncthreads();
  }
  // times the filter spectrum (conjugated for the inverse outer transform)
#pragma unroll
  for (int j = 0; j < E; ++j) {
    const int k = c.tr + j * c.TR;
    C2& x = c.buf[padded<PS>(k)];
    C2 sp = spec[k];
    if (OUTER_INV) sp.y = -sp.y;
    x = cmul(x, sp);
  }
  __syncthreads();
  // inverse FFT_M; the last pass stores the first N outputs
  pow2_load_shared<C2, E, 8, PS>(v, c);
  __syncthreads();
  L = 1;
  lgL = 0;
  for (int p = 0; p < n8; ++p) {
    const bool last = p == n8 - 1 && rem == 0;
    pow2_butterflies<C2, true, E, 8>(v, c, twm, L);
    if (last) {
      blue_store_global<C2, OUTER_INV, E, 8>(v, c, L, lgL, chirp, N);
      return;
    }
    pow2_store<C2, true, E, 8, PS>(v, c, L, lgL, false);
    L <<= 3;
    lgL += 3;
    __syncthreads();
    if (p + 1 < n8) pow2_load_shared<C2, E, 8, PS>(v, c);
    else if (rem == 2) pow2_load_shared<C2, E, 4, PS>(v, c);
    else pow2_load_shared<C2, E, 2, PS>(v, c);
    __syncthreads();
  }
  if (rem == 2) {
    pow2_butterflies<C2, true, E, 4>(v, c, twm, L);
    blue_store_global<C2, OUTER_INV, E, 4>(v, c, L, lgL, chirp, N);
  } else {
    pow2_butterflies<C2, true, E, 2>(v, c, twm, L);
    blue_store_global<C2, OUTER_INV, E, 2>(v, c, L, lgL, chirp, N);
  }
}

// ---- any 7-smooth length ----
// Stockham passes of the plan's radices (8, 4, 2, 3, 5, 7 in the plan's order), one row per
// CTA; each thread takes butterflies t, t + 256, ... of a pass and holds a butterfly's R
// values in registers.  The first pass reads the combined row straight from global memory
// and the last pass writes the row there (L = N / R, so its butterflies store in natural
// order); the passes between exchange values through two shared row buffers.  Twiddles as
// in the power-of-two rows (pass_twiddles); the R-point DFTs of odd R use the symmetric
// form y_m, y_{R-m} = v_0 + sum_s (v_s + v_{R-s}) cos(2 pi s m / R)
// -+ i sum_s (v_s - v_{R-s}) sin(2 pi s m / R) (s = 1 .. (R-1)/2), with the cosines and
// sines of the R-th roots of unity as constants.
// cos(2 pi j / R) and sin(2 pi j / R), 0 <= j <= (R - 1) / 2, R = 3, 5, 7.
__host__ __device__ constexpr double root_cos(int R, int j) {
  return j == 0 ? 1.0
       : R == 3 ? -0.5
       : R == 5 ? (j == 1 ? 0.3090169943749474241023 : -0.8090169943749474241023)
       : (j == 1 ? 0.6234898018587335305250 : j == 2 ? -0.2225209339563144042889 : -0.9009688679024191262361);
}
__host__ __device__ constexpr double root_sin(int R, int j) {
  return j == 0 ? 0.0
       : R == 3 ? 0.8660254037844386467637
       : R == 5 ? (j == 1 ? 0.9510565162951535721164 : 0.5877852522924731291687)
       : (j == 1 ? 0.7818314824680298087084 : j == 2 ? 0.9749279121818236070181 : 0.4338837391175581204758);
}

// y_m = sum_r v_r w_R^{rm}, w_R = exp(-+ 2 pi i / R), R odd.
template <typename C2, bool INV, int R> __device__ __forceinline__ void dft_odd(C2* v) {
  using Re = decltype(v[0].x);
  constexpr int H = (R - 1) / 2;
  C2 sp[H + 1], sm[H + 1];
#pragma unroll
  for (int q = 1; q <= H; ++q) {
    sp[q] = cadd(v[q], v[R - q]);
    sm[q] = csub(v[q], v[R - q]);
  }
  C2 y0 = v[0];
#pragma unroll
  for (int q = 1; q <= H; ++q) y0 = cadd(y0, sp[q]);
#pragma unroll
  for (int m = 1; m <= H; ++m) {
    C2 a = v[0], bsum;
    bsum.x = (Re)0; bsum.y = (Re)0;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      const int j = (q * m) % R;                       // cos, sin of 2 pi j / R
      const int jj = j <= H ? j : R - j;
      const Re cs = (Re)root_cos(R, jj);
      const Re sn = j <= H ? (Re)root_sin(R, jj) : -(Re)root_sin(R, jj);
      a.x += cs * sp[q].x; a.y += cs * sp[q].y;
      bsum.x += sn * sm[q].x; bsum.y += sn * sm[q].y;
    }
    // forward: y_m = a - i bsum, y_{R-m} = a + i bsum; inverse: the other way round
    C2 lo, hi;
    lo.x = a.x + bsum.y; lo.y = a.y - bsum.x;   // a - i bsum
    hi.x = a.x - bsum.y; hi.y = a.y + bsum.x;   // a + i bsum
    v[m] = INV ? hi : lo;
    v[R - m] = INV ? lo : hi;
  }
  v[0] = y0;
}

// Sources and destinations of a pass: the shared buffers, or (first pass) the combined
// input row / (last pass) the output row scaled for the inverse transform.
template <typename C2> struct MixedIO {
  const C2* a;
  const C2* b;     // second source row of the combination or null
  C2 ca, cb;
  int ka, kb, ua, ub;
  C2* o;
  decltype(C2{}.x) scale;
};

template <typename C2, bool INV, int R, bool FIRST, bool LAST>
__device__ __forceinline__ void mixed_pass(const C2* __restrict__ src, C2* __restrict__ dst,
                                           const C2* __restrict__ twp, const MixedIO<C2>& io, int N, int L) {
  const int NR = N / R;
  const float invL = 1.0f / (float)L;
  for (int t = threadIdx.x; t < NR; t += blockDim.x) {
    // j = t / L, k = t mod L (t, L < 2^13: the float quotient is off by at most one)
    int j = (int)((float)t * invL);
    int k = t - j * L;
    if (k >= L) { ++j; k -= L; }
    if (k < 0) { --j; k += L; }
    C2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int i = t + r * NR;
      if (FIRST) {
        C2 x = coef_mul(io.ca, io.ka, io.ua, io.a[i]);
        if (io.b) x = cadd(x, coef_mul(io.cb, io.kb, io.ub, io.b[i]));
        v[r] = x;
      } else {
        v[r] = src[i];
      }
    }
    if (!FIRST) {   // L = 1 in the first pass: no twiddles
      C2 w[R];
      pass_twiddles<C2, R>(w, twp, L, k);
#pragma unroll
      for (int r = 1; r < R; ++r) v[r] = cmul(v[r], conj_if<C2, INV>(w[r]));
    }
    if constexpr (R == 2) dft2<C2, INV>(v);
    else if constexpr (R == 4) dft4<C2, INV>(v);
    else if constexpr (R == 8) dft8<C2, INV>(v);
    else dft_odd<C2, INV, R>(v);
    const int base = j * L * R + k;
#pragma unroll
    for (int s2 = 0; s2 < R; ++s2) {
      if (LAST) {
        C2 y = v[s2];
        y.x *= io.scale;
        y.y *= io.scale;
        io.o[base + s2 * L] = y;
      } else {
        dst[base + s2 * L] = v[s2];
      }
    }
  }
}

template <typename C2, bool INV, bool FIRST, bool LAST>
__device__ __forceinline__ void mixed_pass_r(int Rdx, const C2* src, C2* dst, const C2* __restrict__ twp,
                                             const MixedIO<C2>& io, int N, int L) {
  switch (Rdx) {
    case 2: mixed_pass<C2, INV, 2, FIRST, LAST>(src, dst, twp, io, N, L); break;
    case 3: mixed_pass<C2, INV, 3, FIRST, LAST>(src, dst, twp, io, N, L); break;
    case 4: mixed_pass<C2, INV, 4, FIRST, LAST>(src, dst, twp, io, N, L); break;
    case 5: mixed_pass<C2, INV, 5, FIRST, LAST>(src, dst, twp, io, N, L); break;
    case 7: mixed_pass<C2, INV, 7, FIRST, LAST>(src, dst, twp, io, N, L); break;
    default: mixed_pass<C2, INV, 8, FIRST, LAST>(src, dst, twp, io, N, L); break;
  }
}

template <typename R, bool INV>
__global__ void __launch_bounds__(256) k_fft_rows(const typename Vec2<R>::T* __restrict__ in,
                                                  typename Vec2<R>::T* __restrict__ out,
                                                  const typename Vec2<R>::T* __restrict__ twp, RowCombine rc,
                                                  FftPlan plan, int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = plan.N;
  C2* buf0 = reinterpret_cast<C2*>(smem_raw);
  C2* buf1 = buf0 + N;
  const int row = blockIdx.x;
  const int comp = row / rows_per_comp;
  const int rr = row % rows_per_comp;
  MixedIO<C2> io;
  io.a = in + ((size_t)rc.srcA[comp] * rows_per_comp + rr) * N;
  const int sb = rc.srcB[comp];
  io.b = sb >= 0 ? in + ((size_t)sb * rows_per_comp + rr) * N : nullptr;
  row_coefs<R>(rc, comp, io.ca, io.cb, io.ka, io.kb, io.ua, io.ub);
  io.o = out + (size_t)row * N;
  io.scale = INV ? (R)1 / (R)N : (R)1;
  // radices packed 4 bits each (a parameter array indexed at run time would be copied to
  // the stack)
  unsigned long long radix = 0;
#pragma unroll
  for (int p = 0; p < kMaxRadixPasses; ++p) radix |= (unsigned long long)plan.radix[p] << (4 * p);
  const int np = plan.n_pass;
  if (np == 1) {
    mixed_pass_r<C2, INV, true, true>((int)(radix & 15), buf0, buf1, twp, io, N, 1);
    return;
  }
  mixed_pass_r<C2, INV, true, false>((int)(radix & 15), buf0, buf0, twp, io, N, 1);
  __syncthreads();
  C2* src = buf0;
  C2* dst = buf1;
  int L = (int)(radix & 15);
  for (int p = 1; p < np - 1; ++p) {
    const int Rp = (int)((radix >> (4 * p)) & 15);
    mixed_pass_r<C2, INV, false, false>(Rp, src, dst, twp, io, N, L);
    __syncthreads();
    C2* t2 = src; src = dst; dst = t2;
    L *= Rp;
  }
  mixed_pass_r<C2, INV, false, true>((int)((radix >> (4 * (np - 1))) & 15), src, dst, twp, io, N, L);
}

// ---- any other length: Bluestein's chirp-z algorithm ----
// With w_n = exp(i pi n^2 / N) (n^2 reduced mod 2N in integers, tabulated at set-up),
//   forward: X_k = conj(w_k) sum_n (x_n conj(w_n)) w_{k-n},
//   inverse: x_n = (1/N) w_n sum_k (X_k w_k) conj(w_{n-k}),
// since nk = (n^2 + k^2 - (k-n)^2)/2.  The sums are linear convolutions, done as circular
// ones of power-of-two length M >= 2N - 1: pre-multiply and zero-pad (with the component
// combination on load), FFT_M, multiply by the spectrum S of the filter b (b_m = w_|m| for
// |m| < N, placed mod M; conj(S) for the inverse, as b is even), inverse FFT_M,
// post-multiply -- all in k_fft_blue, one CTA per row (or several short rows).
}  // namespace

int bluestein_length(int Nz, int precision) {
  int n = Nz;
  for (int f : {2, 3, 5, 7})
    while (n > 0 && n % f == 0) n /= f;
  if (n == 1 || Nz < 2) return 0;   // 7-smooth: direct FFT
  int M = 16;
  while (M < 2 * Nz - 1) M <<= 1;
  return M <= (precision == PIC_FP64 ? 4096 : 8192) ? M : 0;
}

// Factor Nz into passes of radix 8, 4, 2, 3, 5, 7 (the Stockham order is free).
bool plan_radix(int N, int32_t* radix, int32_t* n_pass) {
  int n = N, k = 0;
  const int order[6] = {8, 4, 2, 3, 5, 7};
  for (int f : order) {
    while (n % f == 0) {
      if (k >= kMaxRadixPasses) return false;
      radix[k++] = f;
      n /= f;
    }
  }
  *n_pass = k;
  return n == 1;
}

// The shared-memory limit of the FFT kernels is raised once per device to the largest row
// pair any configuration uses (2 x 4096 complex double = 2 x 8192 complex float = 128 KB):
// the attribute is per function, so changing it per launch would race between host
// threads that launch for simulations of different Nz.
constexpr int kFftSmemMax = 2 * 4096 * 16;

pic_status fft_configure_device() {
  static std::mutex mu;
  static bool done[64] = {};
  int dev = 0;
  PIC_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lock(mu);
  if (dev >= 0 && dev < 64 && done[dev]) return PIC_OK;
  PIC_CUDA(cudaFuncSetAttribute(k_fft_rows<double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_rows<double, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_rows<float, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_rows<float, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftSmemMax));
  // power-of-two rows: one padded row buffer (float: staging areas as well)
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2_tma<false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_tma_smem(8192)));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2_tma<true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_tma_smem(8192)));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2_tma<false, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_tma_smem(1024)));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2_tma<true, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fft_tma_smem(1024)));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<double, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<double, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<dw, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<dw, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  // float64 rows of 8192 (one row per CTA, 32 values per thread): 8192 + 1024 padded doubles
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<double, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9216 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<double, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9216 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<dw, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9216 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_pow2<dw, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 9216 * 16));
  // Bluestein rows of length M = 8192 (float) / 4096 (double)
  PIC_CUDA(cudaFuncSetAttribute(k_fft_blue<float, false, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8704 * 8));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_blue<float, true, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize, 8704 * 8));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_blue<double, false, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  PIC_CUDA(cudaFuncSetAttribute(k_fft_blue<double, true, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 4608 * 16));
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

namespace {

template <typename R, bool INV, int E>
void launch_pow2(Sim* s, int N, const void* in, void* out, const void* twp, const RowCombine& rc, int rows,
                 int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  int lgN = 0;
  while ((1 << lgN) < N) ++lgN;
  constexpr int PS = sizeof(R) == 4 ? 4 : 3;
  const int rpc = kFftThreads / (N / E);
  const size_t smem = (size_t)rpc * (N + (N >> PS)) * sizeof(C2);
  const int grid = (rows + rpc - 1) / rpc;
  using G2 = typename GlobalOf<R>::T;
  k_fft_pow2<R, INV, E><<<grid, kFftThreads, smem, s->stream>>>((const G2*)in, (G2*)out, (const C2*)twp, rc, N,
                                                                lgN, rows, rows_per_comp);
}

template <bool INV, int E>
void launch_pow2_tma_e(Sim* s, int N, const void* in, void* out, const void* twp, const RowCombine& rc,
                       int rows_per_comp) {
  int lgN = 0;
  while ((1 << lgN) < N) ++lgN;
  const int G = kFftTmaThreads * E / N;
  const int n_groups = (rows_per_comp + G - 1) / G * rc.n_out;
  const int grid = std::min(n_groups, dht_tc_sm_count() * fft_tma_ctas<E>());
  k_fft_pow2_tma<INV, E><<<grid, kFftTmaThreads, fft_tma_smem(N), s->stream>>>(
      (const float2*)in, (float2*)out, (const float2*)twp, rc, N, lgN, rows_per_comp, rc.n_out, G,
      s->at<int32_t>(s->lay.err));
}

template <bool INV>
void launch_pow2_tma(Sim* s, int N, const void* in, void* out, const void* twp, const RowCombine& rc,
                     int rows_per_comp) {
  if (fft_tma_e(N) == 16) launch_pow2_tma_e<INV, 16>(s, N, in, out, twp, rc, rows_per_comp);
  else launch_pow2_tma_e<INV, 8>(s, N, in, out, twp, rc, rows_per_comp);
}

template <typename R, bool INV>
void launch_pow2_e(Sim* s, int N, const void* in, void* out, const void* twp, const RowCombine& rc, int rows,
                   int rows_per_comp) {
  if (N <= 2048) launch_pow2<R, INV, 8>(s, N, in, out, twp, rc, rows, rows_per_comp);
  else if (N == 4096) launch_pow2<R, INV, 16>(s, N, in, out, twp, rc, rows, rows_per_comp);
  else launch_pow2<R, INV, 32>(s, N, in, out, twp, rc, rows, rows_per_comp);
}

template <typename R, bool INV, int E>
void launch_blue(Sim* s, const void* in, void* out, const RowCombine& rc, int rows, int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  const bool f32 = sizeof(R) == 4;
  const int N = s->cfg.Nz, M = s->blue_M;
  int lgM = 0;
  while ((1 << lgM) < M) ++lgM;
  constexpr int PS = sizeof(R) == 4 ? 4 : 3;
  const int rpc = kFftThreads / (M / E);
  const size_t smem = (size_t)rpc * (M + (M >> PS)) * sizeof(C2);
  const int grid = (rows + rpc - 1) / rpc;
  k_fft_blue<R, INV, E><<<grid, kFftThreads, smem, s->stream>>>(
      (const C2*)in, (C2*)out, s->at<C2>(f32 ? s->lay.twm_f : s->lay.twm), s->at<C2>(f32 ? s->lay.chirp_f : s->lay.chirp),
      s->at<C2>(f32 ? s->lay.bspec_f : s->lay.bspec), rc, N, M, lgM, rows, rows_per_comp);
}

// Bluestein rows: one fused kernel (k_fft_blue), values per thread chosen as for the
// power-of-two rows of length M.
template <typename R, bool INV>
pic_status launch_bluestein(Sim* s, const void* in, void* out, const RowCombine& rc, int rows, int rows_per_comp) {
  const int M = s->blue_M;
  if (M <= 2048) launch_blue<R, INV, 8>(s, in, out, rc, rows, rows_per_comp);
  else if (M == 4096 || sizeof(R) == 8) launch_blue<R, INV, 16>(s, in, out, rc, rows, rows_per_comp);
  else launch_blue<R, INV, sizeof(R) == 8 ? 16 : 32>(s, in, out, rc, rows, rows_per_comp);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace

bool fft_is_pow2(int N) { return N >= 8 && (N & (N - 1)) == 0; }

// Kind, unit and float copies of each combination coefficient (RowCombine).
static void finish_row_combine(RowCombine& rc) {
  auto classify = [](double re, double im, int8_t& kind, int8_t& unit) {
    kind = im == 0.0 ? 0 : (re == 0.0 ? 1 : 2);
    const double v = kind == 0 ? re : im;
    unit = kind < 2 && (v == 1.0 || v == -1.0) ? (v > 0 ? 1 : -1) : 0;
  };
  for (int k = 0; k < 6; ++k) {
    classify(rc.caRe[k], rc.caIm[k], rc.kindA[k], rc.unitA[k]);
    classify(rc.cbRe[k], rc.cbIm[k], rc.kindB[k], rc.unitB[k]);
    rc.fcaRe[k] = (float)rc.caRe[k]; rc.fcaIm[k] = (float)rc.caIm[k];
    rc.fcbRe[k] = (float)rc.cbRe[k]; rc.fcbIm[k] = (float)rc.cbIm[k];
  }
}

pic_status launch_fft_rows(Sim* s, const void* in, void* out, const RowCombine& rc_in, bool inverse) {
  RowCombine rc = rc_in;
  finish_row_combine(rc);
  const pic_config& c = s->cfg;
  const int rows_per_comp = c.Nm * c.Nr;
  const int rows = rc.n_out * rows_per_comp;
  if (s->blue_M > 0) {
    if (c.precision == PIC_FP64)
      return inverse ? launch_bluestein<double, true>(s, in, out, rc, rows, rows_per_comp)
                     : launch_bluestein<double, false>(s, in, out, rc, rows, rows_per_comp);
    return inverse ? launch_bluestein<float, true>(s, in, out, rc, rows, rows_per_comp)
                   : launch_bluestein<float, false>(s, in, out, rc, rows, rows_per_comp);
  }
  if (fft_is_pow2(c.Nz)) {
    if (c.precision == PIC_FP64 && s->dht_path == PIC_DHT_F64_GEMM) {   // IEEE float64 throughout
      const void* twp = s->at<double2>(s->lay.twp);
      if (inverse) launch_pow2_e<double, true>(s, c.Nz, in, out, twp, rc, rows, rows_per_comp);
      else launch_pow2_e<double, false>(s, c.Nz, in, out, twp, rc, rows, rows_per_comp);
    } else if (c.precision == PIC_FP64) {   // double-word butterflies on the float32 units
      const void* twp = s->at<dw2>(s->lay.twp_dw);
      if (inverse) launch_pow2_e<dw, true>(s, c.Nz, in, out, twp, rc, rows, rows_per_comp);
      else launch_pow2_e<dw, false>(s, c.Nz, in, out, twp, rc, rows, rows_per_comp);
    } else {
      const void* twp = s->at<float2>(s->lay.twp_f);
      if (inverse) launch_pow2_tma<true>(s, c.Nz, in, out, twp, rc, rows_per_comp);
      else launch_pow2_tma<false>(s, c.Nz, in, out, twp, rc, rows_per_comp);
    }
    PIC_LAUNCHED(s);
    return PIC_OK;
  }
  FftPlan plan;
  plan.N = c.Nz;
  plan.n_pass = s->n_radix;
  for (int i = 0; i < kMaxRadixPasses; ++i) plan.radix[i] = s->radix[i];
  const double2* tw = s->at<double2>(s->lay.twp);
  const float2* twf = s->at<float2>(s->lay.twp_f);
  const size_t smem = 2 * (size_t)c.Nz * s->cplx_bytes;
  if (c.precision == PIC_FP64) {
    if (inverse) {
      k_fft_rows<double, true><<<rows, 256, smem, s->stream>>>((const double2*)in, (double2*)out, tw, rc,
                                                               plan, rows_per_comp);
    } else {
      k_fft_rows<double, false><<<rows, 256, smem, s->stream>>>((const double2*)in, (double2*)out, tw, rc,
                                                                plan, rows_per_comp);
    }
  } else {
    if (inverse) {
      k_fft_rows<float, true><<<rows, 256, smem, s->stream>>>((const float2*)in, (float2*)out, twf, rc,
                                                              plan, rows_per_comp);
    } else {
      k_fft_rows<float, false><<<rows, 256, smem, s->stream>>>((const float2*)in, (float2*)out, twf, rc,
                                                               plan, rows_per_comp);
    }
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
