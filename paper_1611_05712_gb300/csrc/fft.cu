// Batched complex DFT along z (a5, a9): Fourier transform along z of the
// quasi-cylindrical scheme (section "Finite order pseudo-spectral solvers").
//   forward: Fhat(k) = sum_i F(z_i) e^{-2 pi i k i / Nz}
//   inverse: F(z_i) = (1/Nz) sum_k Fhat(k) e^{+2 pi i k i / Nz}
// One CTA per row; the row is staged in shared memory and transformed by a mixed-radix
// (2, 3, 4, 5, 7) self-sorting Stockham sequence of passes between two shared buffers.
// The component combination of the quasi-cylindrical scheme is fused into the row load:
// out = ca * inA + cb * inB, which forms J_+- = (J_r -+ i J_theta)/2 before the forward
// transform and E_r = E_+ + E_-, E_theta = i (E_+ - E_-) before the inverse one.
#include <mutex>

#include "pic_internal.cuh"

namespace pic {
namespace {

template <typename R> struct Vec2;
template <> struct Vec2<double> { using T = double2; };
template <> struct Vec2<float> { using T = float2; };

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

struct FftPlan {
  int N;
  int n_pass;
  int radix[kMaxRadixPasses];
};

template <typename R, bool INV>
__device__ __forceinline__ typename Vec2<R>::T twiddle(const typename Vec2<R>::T* tw, int idx) {
  typename Vec2<R>::T w;
  const typename Vec2<R>::T t = tw[idx];
  w.x = (R)t.x;
  w.y = INV ? (R)(-t.y) : (R)t.y;
  return w;
}

template <typename R, bool INV>
__global__ void __launch_bounds__(256) k_fft_rows(const typename Vec2<R>::T* __restrict__ in,
                                                  typename Vec2<R>::T* __restrict__ out,
                                                  const typename Vec2<R>::T* __restrict__ tw, RowCombine rc,
                                                  FftPlan plan, int rows_per_comp) {
  using C2 = typename Vec2<R>::T;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int N = plan.N;
  C2* buf0 = reinterpret_cast<C2*>(smem_raw);
  C2* buf1 = buf0 + N;
  const int row = blockIdx.x;
  const int comp = row / rows_per_comp;
  const int rr = row % rows_per_comp;
  const C2* a = in + ((size_t)rc.srcA[comp] * rows_per_comp + rr) * N;
  const int sb = rc.srcB[comp];
  const C2* b = sb >= 0 ? in + ((size_t)sb * rows_per_comp + rr) * N : nullptr;
  C2 ca, cb;
  ca.x = (R)rc.caRe[comp]; ca.y = (R)rc.caIm[comp];
  cb.x = (R)rc.cbRe[comp]; cb.y = (R)rc.cbIm[comp];
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    C2 v = cmul(ca, a[i]);
    if (b) v = cadd(v, cmul(cb, b[i]));
    buf0[i] = v;
  }
  __syncthreads();
  C2* src = buf0;
  C2* dst = buf1;
  int L = 1;
  for (int p = 0; p < plan.n_pass; ++p) {
    const int Rdx = plan.radix[p];
    const int stride = N / Rdx;           // input stride of one butterfly
    const int tstep = stride / L;         // twiddle index step: N/(L*R)
    for (int t = threadIdx.x; t < stride; t += blockDim.x) {
      const int k = t % L;
      const int base = (t / L) * L * Rdx + k;
      C2 v[7];
      for (int r = 0; r < Rdx; ++r) v[r] = src[t + r * stride];
      if (L > 1) {
        for (int r = 1; r < Rdx; ++r) v[r] = cmul(v[r], twiddle<R, INV>(tw, r * k * tstep));
      }
      if (Rdx == 2) {
        C2 y0 = cadd(v[0], v[1]), y1 = csub(v[0], v[1]);
        dst[base] = y0;
        dst[base + L] = y1;
      } else if (Rdx == 4) {
        C2 s02 = cadd(v[0], v[2]), d02 = csub(v[0], v[2]);
        C2 s13 = cadd(v[1], v[3]), d13 = mul_mi<C2, INV>(csub(v[1], v[3]));
        dst[base] = cadd(s02, s13);
        dst[base + L] = cadd(d02, d13);
        dst[base + 2 * L] = csub(s02, s13);
        dst[base + 3 * L] = csub(d02, d13);
      } else {
        // generic small DFT: y_s = sum_r v_r w_R^{r s}, w_R = tw[N/R]
        const int wstep = N / Rdx;
        for (int s = 0; s < Rdx; ++s) {
          C2 acc = v[0];
          for (int r = 1; r < Rdx; ++r) acc = cadd(acc, cmul(v[r], twiddle<R, INV>(tw, ((r * s) % Rdx) * wstep)));
          dst[base + s * L] = acc;
        }
      }
    }
    __syncthreads();
    C2* t2 = src; src = dst; dst = t2;
    L *= Rdx;
  }
  C2* o = out + (size_t)row * N;
  const R scale = INV ? (R)(1.0 / N) : (R)1;
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    C2 v = src[i];
    v.x *= scale;
    v.y *= scale;
    o[i] = v;
  }
}

}  // namespace

// Factor Nz into passes of radix 4, 2, 3, 5, 7 (the Stockham order is free).
bool plan_radix(int N, int32_t* radix, int32_t* n_pass) {
  int n = N, k = 0;
  const int order[5] = {4, 2, 3, 5, 7};
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
  if (dev >= 0 && dev < 64) done[dev] = true;
  return PIC_OK;
}

pic_status launch_fft_rows(Sim* s, const void* in, void* out, const RowCombine& rc, bool inverse) {
  const pic_config& c = s->cfg;
  FftPlan plan;
  plan.N = c.Nz;
  plan.n_pass = s->n_radix;
  for (int i = 0; i < kMaxRadixPasses; ++i) plan.radix[i] = s->radix[i];
  const int rows_per_comp = c.Nm * c.Nr;
  const int rows = rc.n_out * rows_per_comp;
  const double2* tw = s->at<double2>(s->lay.twiddle);
  const float2* twf = s->at<float2>(s->lay.twiddle_f);
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
