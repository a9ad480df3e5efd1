// Setup stage (a0), FP64 on the GPU, once per simulation:
//   * Bessel zeros alpha_{m,n} and k_{m,n} = alpha_{m,n}/R (quasi-cylindrical Hankel grid,
//     section "Finite order pseudo-spectral solvers": Hankel transform along r);
//   * inverse Hankel matrices B_p[j][n] = J_p(k_{m,n} r_j), p = m-1, m, m+1;
//   * forward matrices M_p = pinv(B_p) by a one-sided (Hestenes) Jacobi SVD, dropping
//     singular values <= 1e-3 sigma_max (B_{m-1} lacks the k=0 Dini function);
//   * [k_z]_p from Eq. finite_difference and the [k_z] equation, and the PSATD
//     coefficient tables of Eq. psatd-eqE / psatd-eqB with k_z -> [k_z]_p;
//   * the FFT twiddle table.
#include <math.h>

#include <algorithm>

#include <cuda_bf16.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

// ---------------------------------------------------------------------------------
// Bessel functions of the first kind J_n(x), 0 <= n <= 8, x >= 0, float64.
// x < 1: power series.  1 <= x < 25: Miller's backward recurrence normalised with
// J_0 + 2 sum_k J_2k = 1 (J.C.P. Miller 1952).  x >= 25: Hankel's asymptotic expansion
// J_n(x) = sqrt(2/(pi x)) (P cos chi - Q sin chi), chi = x - (n/2 + 1/4) pi, with
// P, Q the even/odd parts of sum_k a_k(n)/x^k, a_k = prod_{i<=k}(4n^2-(2i-1)^2)/(k! 8^k)
// (Abramowitz & Stegun 9.2.5, 9.2.9-9.2.10), summed while the terms still shrink.
// ---------------------------------------------------------------------------------
__device__ double bessel_series(int n, double x) {
  double h = 0.5 * x, t = 1.0;
  for (int i = 1; i <= n; ++i) t *= h / i;
  double sum = t, h2 = h * h;
  for (int k = 1; k < 30; ++k) {
    t *= -h2 / (k * (double)(k + n));
    sum += t;
    if (fabs(t) < 1e-18 * fabs(sum)) break;
  }
  return sum;
}

__device__ double bessel_miller(int n, double x) {
  int top = 2 * (((int)x + 52) / 2);      // even start order, J_top(x) < 1e-19 for x < 25
  double jp1 = 0.0, j = 1e-30, norm = 0.0, out = 0.0;
  for (int k = top; k >= 1; --k) {
    double jm1 = (2.0 * k / x) * j - jp1;  // J_{k-1}
    jp1 = j;
    j = jm1;
    if (fabs(j) > 1e200) {                 // rescale everything kept so far
      j *= 1e-200; jp1 *= 1e-200; norm *= 1e-200; out *= 1e-200;
    }
    int km1 = k - 1;
    if (km1 == n) out = j;
    if (km1 > 0 && (km1 & 1) == 0) norm += 2.0 * j;
  }
  norm += j;                               // + J_0
  return out / norm;
}

__device__ double bessel_asym(int n, double x) {
  double mu = 4.0 * n * n;
  double term = 1.0, P = 1.0, Q = 0.0, last = 1.0;
  for (int k = 1; k < 60; ++k) {
    double odd = 2.0 * k - 1.0;
    double nt = term * (mu - odd * odd) / (k * 8.0 * x);
    if (fabs(nt) >= fabs(last) && k > 2) break;   // asymptotic: stop at the smallest term
    last = nt;
    term = nt;
    switch (k & 3) {                       // signs: +a0 - a2 + a4 ... ; +a1 - a3 + a5 ...
      case 1: Q += term; break;
      case 2: P -= term; break;
      case 3: Q -= term; break;
      case 0: P += term; break;
    }
    if (fabs(term) < 1e-18) break;
  }
  double s, c;
  sincos(x, &s, &c);
  // chi = x - phi, phi = (2n+1) pi/4: cos/sin phi = +-sqrt(1/2) by n mod 4
  const double h = 0.70710678118654752440;
  double cph, sph;
  switch (n & 3) {
    case 0: cph = h;  sph = h;  break;
    case 1: cph = -h; sph = h;  break;
    case 2: cph = -h; sph = -h; break;
    default: cph = h; sph = -h; break;
  }
  double cchi = c * cph + s * sph;
  double schi = s * cph - c * sph;
  return sqrt(2.0 / (kPi * x)) * (P * cchi - Q * schi);
}

__device__ double bessel_j(int n, double x) {
  double sign = 1.0;
  if (n < 0) {                          // J_{-n} = (-1)^n J_n
    n = -n;
    if (n & 1) sign = -1.0;
  }
  if (x == 0.0) return n == 0 ? sign : 0.0;
  if (x < 1.0) return sign * bessel_series(n, x);
  if (x < 25.0) return sign * bessel_miller(n, x);
  return sign * bessel_asym(n, x);
}

// Zeros alpha_{m,n} (n = 1..Nr) by Newton from McMahon's expansion; kperp = alpha/R.
__global__ void k_bessel_zeros(double* kperp, int Nm, int Nr, double R, int32_t* err) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= Nm * Nr) return;
  int m = idx / Nr, n = idx % Nr + 1;
  double beta = (n + 0.5 * m - 0.25) * kPi;
  double mu = 4.0 * m * m;
  double b8 = 8.0 * beta;
  double x = beta - (mu - 1.0) / b8 - 4.0 * (mu - 1.0) * (7.0 * mu - 31.0) / (3.0 * b8 * b8 * b8);
  bool ok = false;
  for (int it = 0; it < 60; ++it) {
    double f = bessel_j(m, x);
    double fp = (m == 0) ? -bessel_j(1, x) : bessel_j(m - 1, x) - (m / x) * f;
    double dx = f / fp;
    x -= dx;
    if (fabs(dx) <= 1e-15 * x) { ok = true; break; }
  }
  if (!ok) atomicOr(err, kErrTimeout);
  kperp[idx] = x / R;
}

// binv[m][slot][j][n] = J_{m-1+slot}(kperp[m][n] * r_j), r_j = (j + 1/2) dr
__global__ void k_hankel_inv(double* binv, const double* kperp, int Nm, int Nr, double dr) {
  size_t total = (size_t)Nm * 3 * Nr * Nr;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    int n = idx % Nr;
    int j = (idx / Nr) % Nr;
    int slot = (idx / ((size_t)Nr * Nr)) % 3;
    int m = idx / ((size_t)3 * Nr * Nr);
    double r = (j + 0.5) * dr;
    binv[idx] = bessel_j(m - 1 + slot, r * kperp[m * Nr + n]);
  }
}

// ---------------------------------------------------------------------------------
// One-sided Jacobi SVD of all 3 Nm Hankel matrices together.  wt[c][j] = B[j][c] (column
// c stored contiguously), vt[c][i] = V[i][c], initialised to the identity.  Column pairs
// are visited in round-robin order (nn-1 rounds of nn/2 disjoint pairs per sweep); the
// pairs of a round are independent, so one launch per round rotates every pair of every
// matrix at once, one warp per pair.  The host checks after each sweep whether any pair
// was rotated.  At the end d[c] = 1/sigma_c^2 for kept columns, 0 otherwise, so that
// pinv(B)[n][j] = sum_c vt[c][n] wt[c][j] d[c].
// ---------------------------------------------------------------------------------
constexpr int kSvdThreads = 1024;
constexpr int kSvdRoundThreads = 256;
constexpr int kSvdMaxSweeps = 60;

__global__ void k_svd_init(const double* binv, double* wt_all, double* vt_all, int Nr, int nmat) {
  const size_t Nr2 = (size_t)Nr * Nr, total = Nr2 * nmat;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const size_t mat = idx / Nr2;
    const int e = (int)(idx - mat * Nr2);
    const int c = e / Nr, j = e - c * Nr;
    wt_all[idx] = binv[mat * Nr2 + (size_t)j * Nr + c];
    vt_all[idx] = (c == j) ? 1.0 : 0.0;
  }
}

// Pair k of round `round` (nn columns, the padding column of an odd Nr never rotates).
__global__ void __launch_bounds__(kSvdRoundThreads) k_jacobi_round(double* wt_all, double* vt_all, int Nr, int nn,
                                                                  int round, double tol, int32_t* rotated) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (k >= nn / 2) return;
  const size_t off = (size_t)blockIdx.y * Nr * Nr;
  double* wt = wt_all + off;
  double* vt = vt_all + off;
  int p, q;
  if (k == 0) { p = nn - 1; q = round; }
  else { p = (round + k) % (nn - 1); q = (round - k + nn - 1) % (nn - 1); }
  if (p >= Nr || q >= Nr) return;
  if (p > q) { const int t = p; p = q; q = t; }
  double* wp = wt + (size_t)p * Nr;
  double* wq = wt + (size_t)q * Nr;
  double a = 0.0, b = 0.0, g = 0.0;
  for (int j = lane; j < Nr; j += 32) {
    const double x = wp[j], y = wq[j];
    a = fma(x, x, a); b = fma(y, y, b); g = fma(x, y, g);
  }
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
    g += __shfl_xor_sync(0xffffffffu, g, o);
  }
  if (a == 0.0 || b == 0.0 || fabs(g) <= tol * sqrt(a * b)) return;
  const double zeta = (b - a) / (2.0 * g);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
  for (int j = lane; j < Nr; j += 32) {
    const double x = wp[j], y = wq[j];
    wp[j] = c * x - s * y;
    wq[j] = s * x + c * y;
  }
  double* vp = vt + (size_t)p * Nr;
  double* vq = vt + (size_t)q * Nr;
  for (int j = lane; j < Nr; j += 32) {
    const double x = vp[j], y = vq[j];
    vp[j] = c * x - s * y;
    vq[j] = s * x + c * y;
  }
  if (lane == 0) *rotated = 1;
}

// Singular values (column norms of the rotated W) and the cutoff relative to the largest:
// one CTA per matrix.
__global__ void __launch_bounds__(kSvdThreads) k_svd_values(const double* wt_all, double* d_all, int Nr) {
  const int mat = blockIdx.x;
  const double* wt = wt_all + (size_t)mat * Nr * Nr;
  double* d = d_all + (size_t)mat * Nr;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
  __shared__ double smax;
  for (int c = warp; c < Nr; c += nwarps) {
    double a = 0.0;
    for (int j = lane; j < Nr; j += 32) a = fma(wt[(size_t)c * Nr + j], wt[(size_t)c * Nr + j], a);
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) d[c] = a;   // sigma^2 for now
  }
  __syncthreads();
  if (tid == 0) {
    double m2 = 0.0;
    for (int c = 0; c < Nr; ++c) m2 = fmax(m2, d[c]);
    smax = sqrt(m2);
  }
  __syncthreads();
  for (int c = tid; c < Nr; c += blockDim.x) {
    const double sig = sqrt(d[c]);
    d[c] = (sig > kPinvRcond * smax) ? 1.0 / d[c] : 0.0;
  }
}

// mfwd[mat][n][j] = sum_c vt[c][n] wt[c][j] d[c]
__global__ void k_pinv_assemble(const double* wt_all, const double* vt_all, const double* d_all,
                                double* mfwd, int Nr) {
  const int mat = blockIdx.z;
  const double* wt = wt_all + (size_t)mat * Nr * Nr;
  const double* vt = vt_all + (size_t)mat * Nr * Nr;
  const double* d = d_all + (size_t)mat * Nr;
  __shared__ double sv[32][33], sw[32][33];
  int n = blockIdx.y * 32 + threadIdx.y;
  int j = blockIdx.x * 32 + threadIdx.x;
  double acc = 0.0;
  for (int c0 = 0; c0 < Nr; c0 += 32) {
    int c = c0 + threadIdx.x;
    int nn = blockIdx.y * 32 + threadIdx.y;
    sv[threadIdx.y][threadIdx.x] = (c < Nr && nn < Nr) ? vt[(size_t)c * Nr + nn] * d[c] : 0.0;
    int cc = c0 + threadIdx.y;
    sw[threadIdx.y][threadIdx.x] = (cc < Nr && j < Nr) ? wt[(size_t)cc * Nr + j] : 0.0;
    __syncthreads();
    for (int k = 0; k < 32; ++k) acc = fma(sv[threadIdx.y][k], sw[k][threadIdx.x], acc);
    __syncthreads();
  }
  if (n < Nr && j < Nr) mfwd[((size_t)mat * Nr + n) * Nr + j] = acc;
}

// w[mat][i][j] = 2 delta_ij - w[mat][i][j]
__global__ void k_two_minus(double* w, int nmat, int Nr) {
  const size_t total = (size_t)nmat * Nr * Nr;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int j = idx % Nr, i = (idx / Nr) % Nr;
    w[idx] = (i == j ? 2.0 : 0.0) - w[idx];
  }
}

// [k_z]_p per FFT bin: k_z = 2 pi f/(Nz dz), f in FFT order (Nyquist negative);
// [k_z] = sum_{j=1}^{n} alpha_{n,j} sin(k_z j dz)/(j dz), p = 2n; p = 0 -> k_z.
// Filter factor Tz = cos^2(k_z dz/2) (exact k_z).
__global__ void k_kz_tables(double* kzmod, double* tz, int Nz, double dz, int order_p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Nz) return;
  int f = (i < (Nz + 1) / 2) ? i : i - Nz;
  double kz = (2.0 * kPi) * ((double)f * (1.0 / (Nz * dz)));
  double km = kz;
  if (order_p > 0) {
    int n = order_p / 2;
    double prod = 1.0;
    km = 0.0;
    for (int j = 1; j <= n; ++j) {
      prod *= (double)(n - j + 1) / (double)(n + j);
      double alpha = ((j & 1) ? 2.0 : -2.0) * prod;
      km += alpha * sin(kz * (j * dz)) / (j * dz);
    }
  }
  kzmod[i] = km;
  double c = cos(0.5 * kz * dz);
  tz[i] = c * c;
}

__global__ void k_tr_table(double* tr, const double* kperp, int n, double dr) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double c = cos(0.5 * kperp[i] * dr);
  tr[i] = c * c;
}

// Per spectral cell (m, n, kz), SI (Eq. psatd-eqE/eqB with [k_z]):
//   coef[0] = C = cos(x), coef[1] = S/K, coef[2] = (1-C)/K^2 = 2 sin^2(x/2)/K^2,
//   coef[3] = (S/x - 1)/K^2, coef[4] = (C - S/x)/K^2, coef[5] = 1/K^2,
// with K^2 = k_perp^2 + [k_z]^2, x = c K dt; coef[3], coef[4] by power series for x < 0.25.
__global__ void k_psatd_coef(double* coef, const double* kperp, const double* kzmod, int Nm, int Nr,
                             int Nz, double dt) {
  size_t G = (size_t)Nm * Nr * Nz;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    int kz = idx % Nz;
    size_t mn = idx / Nz;
    double Kp = kperp[mn], Kz = kzmod[kz];
    double K2 = Kp * Kp + Kz * Kz;
    double K = sqrt(K2);
    double cdt = kC * dt;
    double x = cdt * K;
    double s, c, sh, ch;
    sincos(x, &s, &c);
    sincos(0.5 * x, &sh, &ch);
    double an, ap;
    if (x < kSmallX) {
      // (sin x - x)/x = sum_{k>=1} (-1)^k x^{2k}/(2k+1)!,
      // (x cos x - sin x)/x = sum_{k>=1} (-1)^k x^{2k} 2k/(2k+1)!; divided by K^2 = x^2/cdt^2.
      double x2 = x * x, pw = 1.0, fact = 6.0;   // fact = (2k+1)!
      an = 0.0; ap = 0.0;
      for (int k = 1; k < 10; ++k) {
        double sg = (k & 1) ? -1.0 : 1.0;
        an += sg * pw / fact;
        ap += sg * (2.0 * k) * pw / fact;
        pw *= x2;
        fact *= (2.0 * k + 2.0) * (2.0 * k + 3.0);
      }
      an *= cdt * cdt;
      ap *= cdt * cdt;
    } else {
      an = (s / x - 1.0) / K2;
      ap = (c - s / x) / K2;
    }
    coef[0 * G + idx] = c;
    coef[1 * G + idx] = s / K;
    coef[2 * G + idx] = 2.0 * sh * sh / K2;
    coef[3 * G + idx] = an;
    coef[4 * G + idx] = ap;
    coef[5 * G + idx] = 1.0 / K2;
  }
}

// tw[k] = exp(-2 pi i k / N), k < N
// Power-of-two Nz: twiddles of the radix-8 Stockham passes (radix R, L = product of the
// earlier radices): entry L-1 + (r-1) L + k holds w_{LR}^{rk} = exp(-2 pi i r k / (L R)),
// 1 <= r < R, k < L; the passes' tables tile entries 0..N-2 (entry N-1 is unused).
__global__ void k_twiddles_pow2(double2* tw, int N) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  if (idx == N - 1) { tw[idx] = make_double2(1.0, 0.0); return; }
  int lgN = 0;
  while ((1 << lgN) < N) ++lgN;
  const int n8 = lgN / 3, rem = lgN - 3 * n8;
  int L = 1;
  for (int p = 0; p < n8 + (rem ? 1 : 0); ++p) {
    const int R = p < n8 ? 8 : (1 << rem);
    if (idx < L - 1 + (R - 1) * L) {
      const int off = idx - (L - 1);
      const int r = off / L + 1, k = off % L;
      double sn, cs;
      sincospi(2.0 * (double)(r * k) / (double)(L * R), &sn, &cs);
      tw[idx] = make_double2(cs, -sn);
      return;
    }
    L *= R;
  }
}

// Any 7-smooth Nz: twiddles of the mixed-radix Stockham passes radix[0], radix[1], ...
// (the plan of the row FFT), at the same entries: pass p (radix R, L = product of the
// earlier radices) holds w_{LR}^{rk} at L-1 + (r-1) L + k.
struct RadixPlan {
  int n_pass;
  int radix[kMaxRadixPasses];
};

__global__ void k_twiddles_plan(double2* tw, int N, RadixPlan plan) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= N) return;
  if (idx == N - 1) { tw[idx] = make_double2(1.0, 0.0); return; }
  int L = 1;
  for (int p = 0; p < plan.n_pass; ++p) {
    const int R = plan.radix[p];
    if (idx < L - 1 + (R - 1) * L) {
      const int off = idx - (L - 1);
      const int r = off / L + 1, k = off % L;
      double sn, cs;
      sincospi(2.0 * (double)(r * k) / (double)(L * R), &sn, &cs);
      tw[idx] = make_double2(cs, -sn);
      return;
    }
    L *= R;
  }
}

inline int blocks_for(size_t n, int t) { return (int)((n + t - 1) / t); }

// float copies of FP64 tables (round to nearest)
__global__ void k_to_float(const double* __restrict__ in, float* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (float)in[i];
}

// x -> (hi, lo) = (float(x), float(x - hi)): a double word of about 48 bits.
__global__ void k_to_double_word(const double* __restrict__ in, float2* __restrict__ out, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const double x = in[i];
    const float h = (float)x;
    out[i] = make_float2(h, (float)(x - (double)h));
  }
}

// Split of FP64 matrices (rows of Nr) for 3-term TF32 products: hi = the value rounded to
// TF32 (10 explicit mantissa bits, low 13 bits of the float zero), lo = float(value - hi).
// Output rows have a pitch of `pitch` >= Nr floats (16-byte multiple for the tensor-memory
// copies); the padding is zero.
__global__ void k_split_tf32(const double* __restrict__ in, float* __restrict__ hi, float* __restrict__ lo,
                             size_t rows, int Nr, int pitch) {
  const size_t n = rows * (size_t)pitch;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(o % pitch);
    if (col >= Nr) { hi[o] = 0.f; lo[o] = 0.f; continue; }
    const double v = in[(o / pitch) * Nr + col];
    const float f = (float)v;
    // round-to-nearest-even at bit 13 of the float's bit pattern (finite values)
    uint32_t b = __float_as_uint(f);
    b = (b + 0x0fffu + ((b >> 13) & 1u)) & 0xffffe000u;
    const float h = __uint_as_float(b);
    hi[o] = h;
    lo[o] = (float)(v - (double)h);
  }
}

// Split of FP64 matrices (rows of Nr) into three BF16 pieces for the BF16 form:
// b0 = bf16(a), b1 = bf16(a - b0), b2 = bf16(a - b0 - b1) (differences in FP64), stored as
// three planes of rows with a pitch of `pitch` >= Nr elements (16-byte multiple); the
// padding is zero.
__global__ void k_split_bf16x3(const double* __restrict__ in, __nv_bfloat16* __restrict__ p0,
                               __nv_bfloat16* __restrict__ p1, __nv_bfloat16* __restrict__ p2, size_t rows,
                               int Nr, int pitch) {
  const size_t n = rows * (size_t)pitch;
  for (size_t o = blockIdx.x * (size_t)blockDim.x + threadIdx.x; o < n; o += (size_t)gridDim.x * blockDim.x) {
    const int col = (int)(o % pitch);
    double v = col < Nr ? in[(o / pitch) * Nr + col] : 0.0;
    const __nv_bfloat16 b0 = __double2bfloat16(v);
    v -= (double)__bfloat162float(b0);
    const __nv_bfloat16 b1 = __double2bfloat16(v);
    v -= (double)__bfloat162float(b1);
    p0[o] = b0;
    p1[o] = b1;
    p2[o] = __double2bfloat16(v);
  }
}

inline int conv_grid(size_t n) { return (int)std::min<size_t>(blocks_for(n, 256), 152 * 16); }

}  // namespace

// Mixed form: float copies of k_perp, the filter factor in r and the split DHT matrices.
pic_status convert_hankel_tables(Sim* s) {
  const pic_config& c = s->cfg;
  const size_t nmn = (size_t)c.Nm * c.Nr, rows = (size_t)c.Nm * 3 * c.Nr;
  const int pitch = split_pitch(c.Nr);
  const size_t nmat = rows * pitch;
  k_to_float<<<conv_grid(nmn), 256, 0, s->stream>>>(s->at<double>(s->lay.kperp), s->at<float>(s->lay.kperp_f), nmn);
  PIC_LAUNCHED(s);
  k_to_float<<<conv_grid(nmn), 256, 0, s->stream>>>(s->at<double>(s->lay.tr), s->at<float>(s->lay.tr_f), nmn);
  PIC_LAUNCHED(s);
  if (c.precision == PIC_MIXED_BF16X6) {
    const int pb = split_pitch_b16(c.Nr);
    const size_t plane = rows * pb;
    for (int dir = 0; dir < 2; ++dir) {
      __nv_bfloat16* base = s->at<__nv_bfloat16>(dir == 0 ? s->lay.mfwd_hi : s->lay.binv_hi);
      k_split_bf16x3<<<conv_grid(plane), 256, 0, s->stream>>>(s->at<double>(dir == 0 ? s->lay.mfwd : s->lay.binv),
                                                               base, base + plane, base + 2 * plane, rows, c.Nr, pb);
      PIC_LAUNCHED(s);
    }
    return PIC_OK;
  }
  k_split_tf32<<<conv_grid(nmat), 256, 0, s->stream>>>(s->at<double>(s->lay.mfwd), s->at<float>(s->lay.mfwd_hi),
                                                         s->at<float>(s->lay.mfwd_lo), rows, c.Nr, pitch);
  PIC_LAUNCHED(s);
  k_split_tf32<<<conv_grid(nmat), 256, 0, s->stream>>>(s->at<double>(s->lay.binv), s->at<float>(s->lay.binv_hi),
                                                         s->at<float>(s->lay.binv_lo), rows, c.Nr, pitch);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

// Mixed form: float copies of the PSATD coefficient tables, [k_z]_p and the z filter.
pic_status convert_psatd_tables(Sim* s) {
  const pic_config& c = s->cfg;
  const size_t G6 = 6 * s->grid_elems();
  k_to_float<<<conv_grid(G6), 256, 0, s->stream>>>(s->at<double>(s->lay.coef), s->at<float>(s->lay.coef_f), G6);
  PIC_LAUNCHED(s);
  k_to_float<<<conv_grid(c.Nz), 256, 0, s->stream>>>(s->at<double>(s->lay.kzmod), s->at<float>(s->lay.kzmod_f), c.Nz);
  PIC_LAUNCHED(s);
  k_to_float<<<conv_grid(c.Nz), 256, 0, s->stream>>>(s->at<double>(s->lay.tz), s->at<float>(s->lay.tz_f), c.Nz);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_setup_hankel(Sim* s) {
  const pic_config& c = s->cfg;
  const int Nm = c.Nm, Nr = c.Nr;
  double* kperp = s->at<double>(s->lay.kperp);
  double* binv = s->at<double>(s->lay.binv);
  int32_t* err = s->at<int32_t>(s->lay.err);
  k_bessel_zeros<<<blocks_for((size_t)Nm * Nr, 128), 128, 0, s->stream>>>(kperp, Nm, Nr, Nr * c.dr, err);
  PIC_LAUNCHED(s);
  size_t tot = (size_t)Nm * 3 * Nr * Nr;
  k_hankel_inv<<<(int)std::min<size_t>(blocks_for(tot, 256), 152 * 16), 256, 0, s->stream>>>(
      binv, kperp, Nm, Nr, c.dr);
  PIC_LAUNCHED(s);
  double* wt = s->at<double>(s->lay.svd_w);
  double* vt = s->at<double>(s->lay.svd_v);
  double* d = s->at<double>(s->lay.svd_d);
  // rotate while |w_p.w_q| > tol |w_p||w_q|; the computed dot product carries a rounding
  // floor of about eps*sqrt(Nr), so the threshold sits above it
  double tol = 2e-15 * std::sqrt((double)Nr);
  const int nmat = Nm * 3, nn = Nr + (Nr & 1);
  k_svd_init<<<(int)std::min<size_t>(blocks_for((size_t)nmat * Nr * Nr, 256), 152 * 16), 256, 0, s->stream>>>(
      binv, wt, vt, Nr, nmat);
  PIC_LAUNCHED(s);
  // the sort's counter word is free during set-up: it records whether a sweep rotated
  int32_t* rotated = s->at<int32_t>(s->lay.big_count);
  const dim3 rgrid((unsigned)blocks_for((size_t)(nn / 2) * 32, kSvdRoundThreads), (unsigned)nmat);
  bool converged = false;
  for (int sweep = 0; sweep < kSvdMaxSweeps && !converged; ++sweep) {
    PIC_CUDA(cudaMemsetAsync(rotated, 0, sizeof(int32_t), s->stream));
    for (int round = 0; round < nn - 1; ++round) {
      k_jacobi_round<<<rgrid, kSvdRoundThreads, 0, s->stream>>>(wt, vt, Nr, nn, round, tol, rotated);
      PIC_LAUNCHED(s);
    }
    int32_t h = 1;
    PIC_CUDA(cudaMemcpyAsync(&h, rotated, sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    PIC_CUDA(cudaStreamSynchronize(s->stream));
    converged = h == 0;
  }
  if (!converged) {
    set_error("Jacobi SVD of the Hankel matrices did not converge in %d sweeps", kSvdMaxSweeps);
    return PIC_ERR_TIMEOUT;
  }
  k_svd_values<<<nmat, kSvdThreads, 0, s->stream>>>(wt, d, Nr);
  PIC_LAUNCHED(s);
  double* mfwd = s->at<double>(s->lay.mfwd);
  dim3 g(blocks_for(Nr, 32), blocks_for(Nr, 32), Nm * 3);
  k_pinv_assemble<<<g, dim3(32, 32), 0, s->stream>>>(wt, vt, d, mfwd, Nr);
  PIC_LAUNCHED(s);
  // One Newton-Schulz step M <- M (2I - B M): the Jacobi result is accurate to about
  // tol * cond; the step squares the error on the kept subspace, while components along
  // dropped directions (of size ~tol |M|) only double.  W and V are free again here.
  const size_t Nr2 = (size_t)Nr * Nr;
  DhtBatch bm{}, mt{};
  for (int k = 0; k < Nm * 3; ++k) {
    bm.A[k] = binv + k * Nr2; bm.X[k] = mfwd + k * Nr2; bm.Y[k] = wt + k * Nr2;
    mt.A[k] = mfwd + k * Nr2; mt.X[k] = wt + k * Nr2; mt.Y[k] = vt + k * Nr2;
  }
  bm.n = mt.n = Nm * 3;
  pic_status st = launch_gemm_f64(s, bm, Nr);          // W = B M
  if (st != PIC_OK) return st;
  k_two_minus<<<(int)std::min<size_t>(blocks_for(Nm * 3 * Nr2, 256), 152 * 16), 256, 0, s->stream>>>(
      wt, Nm * 3, Nr);                                  // W = 2I - W
  PIC_LAUNCHED(s);
  if ((st = launch_gemm_f64(s, mt, Nr)) != PIC_OK) return st;   // V = M W
  PIC_CUDA(cudaMemcpyAsync(mfwd, vt, Nm * 3 * Nr2 * sizeof(double), cudaMemcpyDeviceToDevice, s->stream));
  k_tr_table<<<blocks_for((size_t)Nm * Nr, 128), 128, 0, s->stream>>>(s->at<double>(s->lay.tr), kperp,
                                                                       Nm * Nr, c.dr);
  PIC_LAUNCHED(s);
  if (c.precision != PIC_FP64) return convert_hankel_tables(s);
  return launch_f64s_setup(s);
}

pic_status launch_setup_tables(Sim* s, int32_t order_p) {
  const pic_config& c = s->cfg;
  k_kz_tables<<<blocks_for(c.Nz, 128), 128, 0, s->stream>>>(s->at<double>(s->lay.kzmod),
                                                             s->at<double>(s->lay.tz), c.Nz, c.dz,
                                                             order_p);
  PIC_LAUNCHED(s);
  size_t G = s->grid_elems();
  k_psatd_coef<<<(int)std::min<size_t>(blocks_for(G, 256), 152 * 32), 256, 0, s->stream>>>(
      s->at<double>(s->lay.coef), s->at<double>(s->lay.kperp), s->at<double>(s->lay.kzmod), c.Nm,
      c.Nr, c.Nz, c.dt);
  PIC_LAUNCHED(s);
  s->order_tables = order_p;
  if (c.precision != PIC_FP64) return convert_psatd_tables(s);
  return PIC_OK;
}

// Bluestein tables for an Nz that is not 7-smooth: the chirp w_n = exp(i pi t / N) with
// t = n^2 mod 2N computed in integers, and the spectrum of the even filter b (b_m = w_|m| for
// |m| < N, indices mod M): S_k = 1 + 2 sum_{j=1}^{N-1} w_j cos(2 pi (jk mod M) / M), summed
// directly in float64 (once per handle; the arguments 2t/M are exact for M a power of two).
__global__ void k_blue_chirp(double2* chirp, int N) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= N) return;
  const long long t = ((long long)n * n) % (2LL * N);
  double sn, cs;
  sincospi((double)t / (double)N, &sn, &cs);
  chirp[n] = make_double2(cs, sn);
}

__global__ void k_blue_spectrum(const double2* __restrict__ chirp, double2* spec, int N, int M) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= M) return;
  double re = 0.0, im = 0.0;
  for (int j = 1; j < N; ++j) {
    const long long t = ((long long)j * k) & (M - 1);
    const double c = cospi(2.0 * (double)t / (double)M);
    re = fma(chirp[j].x, c, re);
    im = fma(chirp[j].y, c, im);
  }
  spec[k] = make_double2(1.0 + 2.0 * re, 2.0 * im);
}

pic_status launch_setup_twiddles(Sim* s) {
  if (s->blue_M > 0) {
    const int N = s->cfg.Nz, M = s->blue_M;
    k_twiddles_pow2<<<blocks_for(M, 128), 128, 0, s->stream>>>(s->at<double2>(s->lay.twm), M);
    PIC_LAUNCHED(s);
    k_blue_chirp<<<blocks_for(N, 128), 128, 0, s->stream>>>(s->at<double2>(s->lay.chirp), N);
    PIC_LAUNCHED(s);
    k_blue_spectrum<<<blocks_for(M, 128), 128, 0, s->stream>>>(s->at<double2>(s->lay.chirp),
                                                                s->at<double2>(s->lay.bspec), N, M);
    PIC_LAUNCHED(s);
    if (s->cfg.precision != PIC_FP64) {
      const size_t pairs[3][3] = {{s->lay.twm, s->lay.twm_f, 2 * (size_t)M},
                                  {s->lay.chirp, s->lay.chirp_f, 2 * (size_t)N},
                                  {s->lay.bspec, s->lay.bspec_f, 2 * (size_t)M}};
      for (const auto& q : pairs) {
        k_to_float<<<conv_grid(q[2]), 256, 0, s->stream>>>(s->at<double>(q[0]), s->at<float>(q[1]), q[2]);
        PIC_LAUNCHED(s);
      }
    }
    return PIC_OK;
  }
  const bool pow2 = fft_is_pow2(s->cfg.Nz);
  if (pow2) {
    k_twiddles_pow2<<<blocks_for(s->cfg.Nz, 128), 128, 0, s->stream>>>(s->at<double2>(s->lay.twp), s->cfg.Nz);
  } else {
    RadixPlan plan{s->n_radix, {}};
    for (int i = 0; i < kMaxRadixPasses; ++i) plan.radix[i] = s->radix[i];
    k_twiddles_plan<<<blocks_for(s->cfg.Nz, 128), 128, 0, s->stream>>>(s->at<double2>(s->lay.twp), s->cfg.Nz, plan);
  }
  PIC_LAUNCHED(s);
  const size_t n2 = 2 * (size_t)s->cfg.Nz;
  if (s->cfg.precision != PIC_FP64) {
    k_to_float<<<conv_grid(n2), 256, 0, s->stream>>>(s->at<double>(s->lay.twp), s->at<float>(s->lay.twp_f), n2);
  } else {   // double words for the FP64 rows: hi = float(x), lo = float(x - hi)
    k_to_double_word<<<conv_grid(n2), 256, 0, s->stream>>>(s->at<double>(s->lay.twp), s->at<float2>(s->lay.twp_dw),
                                                           n2);
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

bool eb_dw_active(const Sim* s) {
  return s->lay.ebdw != 0 && s->blue_M == 0 && s->dht_path != PIC_DHT_F64_GEMM;
}

pic_status refresh_eb_dw(Sim* s) {
  const size_t n = 12 * s->grid_elems();   // 6 complex planes of float64
  k_to_double_word<<<conv_grid(n), 256, 0, s->stream>>>(s->at<double>(s->lay.E), s->at<float2>(s->lay.ebdw), n);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
