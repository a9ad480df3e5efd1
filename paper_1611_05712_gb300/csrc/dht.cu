// Discrete Hankel transform along r (a6 forward, a8 inverse): for every (component,
// mode) pair, Y = A X with A a real Nr x Nr matrix (pinv(B_p) forward, B_p inverse;
// section "Finite order pseudo-spectral solvers": Hankel transform along r) and X the
// Nr x Nz complex panel of that component seen as Nr x 2Nz reals (re, im interleaved).
//
// FP64 form: register-tiled SIMT GEMM (64 x 64 tile per CTA, 4 x 4 outputs per thread,
// K staged through shared memory in steps of 16).  On GB300 the FP64 pipe, not HBM or
// shared memory, bounds this kernel, so the tile only has to keep that pipe fed.  The same
// kernel serves the FP64 setup products (Newton-Schulz refinement of the pseudo-inverse).
#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int BM = 64, BN = 64, BK = 16;

template <typename R>
__global__ void __launch_bounds__(256) k_gemm(DhtBatch bt, int Nr, int Nc) {
  const int b = blockIdx.z;
  const R* __restrict__ A = static_cast<const R*>(bt.A[b]);
  const R* __restrict__ X = static_cast<const R*>(bt.X[b]);
  R* __restrict__ Y = static_cast<R*>(bt.Y[b]);
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  __shared__ __align__(16) R As[BK][BM];
  __shared__ __align__(16) R Xs[BK][BN];
  const int t = threadIdx.x;
  const int tx = t & 15, ty = t >> 4;
  R acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = (R)0;

  for (int k0 = 0; k0 < Nr; k0 += BK) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = t >> 2, kk = ((t & 3) << 2) + q;
      const int gr = row0 + r, gk = k0 + kk;
      As[kk][r] = (gr < Nr && gk < Nr) ? A[(size_t)gr * Nr + gk] : (R)0;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int kk = t >> 4, cc = ((t & 15) << 2) + q;
      const int gk = k0 + kk, gc = col0 + cc;
      Xs[kk][cc] = (gk < Nr && gc < Nc) ? X[(size_t)gk * Nc + gc] : (R)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      R a[4], x[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
      for (int j = 0; j < 4; ++j) x[j] = Xs[kk][tx * 4 + j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], x[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + ty * 4 + i;
    if (gr >= Nr) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gc = col0 + tx * 4 + j;
      if (gc < Nc) Y[(size_t)gr * Nc + gc] = acc[i][j];
    }
  }
}

}  // namespace

pic_status launch_gemm_f64(Sim* s, const DhtBatch& b, int ncols) {
  const int Nr = s->cfg.Nr;
  dim3 grid((ncols + BN - 1) / BN, (Nr + BM - 1) / BM, b.n);
  k_gemm<double><<<grid, 256, 0, s->stream>>>(b, Nr, ncols);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_dht(Sim* s, const DhtBatch& b) {
  if (s->cfg.precision == PIC_FP64)
    return f64s_active(s) ? launch_dht_f64s(s, b) : launch_gemm_f64(s, b, 2 * s->cfg.Nz);
  return launch_dht_tc(s, b);   // mixed forms: split products on tcgen05 (dht_tc.cu)
}

}  // namespace pic
