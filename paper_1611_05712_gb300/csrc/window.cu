// Moving window, field side: removal of the departing z column from E and B.
//
// The paper follows its beams in the co-moving frame zeta = z - c t (section "Accurate
// modeling of plasma accelerators in finite order PSATD", Fig. ez) without giving the
// mechanics.  Here the z grid is a ring of columns and the window's back column c leaves
// when the window moves: its real-space E and B become zero and the forward transform of
// that column is subtracted from the spectral state,
//     F^_{+-,z}[m][n][k] -= (M_p F_col_{+-,z}[m])[n] * exp(-2 pi i k c / Nz),
// the z-DFT of a single column being the column times one phase per frequency bin
// (forward DFT exp(-i k_z z), no normalisation), and M_p the forward Hankel matrix of order
// p = m+1 (+), m-1 (-), m (z).  Two kernels at the end of the cycle: take the column (with
// F_+- = (F_r -/+ i F_th)/2) and zero it in real space; apply M_p (one warp per output) and
// tabulate the phases.  The subtraction itself is left pending and done by the next PSATD
// update as it loads the spectral fields (no extra pass over them); a call that reads or
// changes the spectral fields before then applies it on its own (launch_window_flush).
#include <math.h>

#include "pic_internal.cuh"

namespace pic {
namespace {

constexpr int kWinThreads = 256;

// colv[(f*3 + c)*Nm + m][j], f = E, B; c = +, -, z.  Grid: 2*Nm*Nr threads.  EBdw, when
// given, is the double-word copy of E, B (same layout, float4 elements): its column is
// zeroed as well.
template <typename T2>
__global__ void k_win_col_take(T2* EB, size_t G, int Nm, int Nr, int Nz, int column, double2* colv,
                               float4* EBdw) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * Nm * Nr) return;
  const int f = t / (Nm * Nr), mj = t - f * Nm * Nr;
  T2* base = EB + (size_t)f * 3 * G + (size_t)mj * Nz + column;   // [f*3 + comp][m][j][column]
  const T2 a = base[0], b = base[G], z = base[2 * G];
  const double ar = a.x, ai = a.y, br = b.x, bi = b.y;
  double2* out = colv + (size_t)f * 3 * Nm * Nr + mj;
  out[0] = make_double2(0.5 * (ar + bi), 0.5 * (ai - br));                 // (F_r - i F_th)/2
  out[(size_t)Nm * Nr] = make_double2(0.5 * (ar - bi), 0.5 * (ai + br));   // (F_r + i F_th)/2
  out[2 * (size_t)Nm * Nr] = make_double2((double)z.x, (double)z.y);
  T2 zero;
  zero.x = 0;
  zero.y = 0;
  base[0] = zero;
  base[G] = zero;
  base[2 * G] = zero;
  if (EBdw) {
    float4* bdw = EBdw + (size_t)f * 3 * G + (size_t)mj * Nz + column;
    const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
    bdw[0] = z4;
    bdw[G] = z4;
    bdw[2 * G] = z4;
  }
}

// hv[row][n] = sum_j M[m][slot][n][j] colv[row][j] with row = (f*3 + c)*Nm + m; the
// blocks past the last output tabulate ph[k] = exp(-2 pi i ((k * column) mod Nz) / Nz)
// (the reduction done in integers).
// Both are also written rounded to float (hvf, phf) for the mixed form.
__global__ void k_win_col_hankel(const double* __restrict__ mfwd, int Nm, int Nr, const double2* __restrict__ colv,
                                 double2* hv, int hankel_blocks, double2* ph, int Nz, int column, float2* hvf,
                                 float2* phf) {
  if ((int)blockIdx.x >= hankel_blocks) {
    const int k = (blockIdx.x - hankel_blocks) * blockDim.x + threadIdx.x;
    if (k < Nz) {
      const long long t = ((long long)k * column) % Nz;
      double sn, cs;
      sincospi(-2.0 * (double)t / (double)Nz, &sn, &cs);
      ph[k] = make_double2(cs, sn);
      phf[k] = make_float2((float)cs, (float)sn);
    }
    return;
  }
  const int lane = threadIdx.x & 31;
  const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;   // one warp per output
  if (o >= 6 * Nm * Nr) return;
  const int row = o / Nr, n = o - row * Nr;
  const int c = (row / Nm) % 3, m = row % Nm;
  const int slot = c == 0 ? 2 : (c == 1 ? 0 : 1);   // +: order m+1, -: m-1, z: m
  const double* a = mfwd + ((size_t)m * 3 + slot) * Nr * Nr + (size_t)n * Nr;
  const double2* x = colv + (size_t)row * Nr;
  double re = 0.0, im = 0.0;
  for (int j = lane; j < Nr; j += 32) {
    re = fma(a[j], x[j].x, re);
    im = fma(a[j], x[j].y, im);
  }
  for (int d = 16; d > 0; d >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, d);
    im += __shfl_xor_sync(0xffffffffu, im, d);
  }
  if (lane == 0) {
    hv[o] = make_double2(re, im);
    hvf[o] = make_float2((float)re, (float)im);
  }
}

// Fh[row][k] -= hv[row] ph[k] over the 6*Nm*Nr spectral rows of E and B (adjacent): the
// pending subtraction applied on its own (same arithmetic as the fused PSATD path).
__global__ void k_win_col_apply64(double2* Fh, int Nz, const double2* __restrict__ hv, const double2* __restrict__ ph) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nz) return;
  const double2 h = hv[blockIdx.y], p = ph[k];
  double2* f = Fh + (size_t)blockIdx.y * Nz + k;
  double2 v = *f;
  v.x -= h.x * p.x - h.y * p.y;
  v.y -= h.x * p.y + h.y * p.x;
  *f = v;
}

__global__ void k_win_col_apply32(float2* Fh, int Nz, const float2* __restrict__ hv, const float2* __restrict__ ph) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= Nz) return;
  const float2 h = hv[blockIdx.y], p = ph[k];
  const float hx = h.x, hy = h.y, px = p.x, py = p.y;
  float2* f = Fh + (size_t)blockIdx.y * Nz + k;
  float2 v = *f;
  v.x -= hx * px - hy * py;
  v.y -= hx * py + hy * px;
  *f = v;
}

}  // namespace

pic_status launch_window_flush(Sim* s) {
  WindowState& w = s->win;
  if (!w.pending) return PIC_OK;
  w.pending = 0;
  const pic_config& c = s->cfg;
  const double2* hv = reinterpret_cast<const double2*>(w.ws + w.hv);
  const double2* ph = reinterpret_cast<const double2*>(w.ws + w.ph);
  const dim3 grid((c.Nz + kWinThreads - 1) / kWinThreads, 6 * c.Nm * c.Nr);
  if (c.precision == PIC_FP64)
    k_win_col_apply64<<<grid, kWinThreads, 0, s->stream>>>(s->at<double2>(s->lay.Eh), c.Nz, hv, ph);
  else
    k_win_col_apply32<<<grid, kWinThreads, 0, s->stream>>>(s->at<float2>(s->lay.Eh), c.Nz,
                                                            reinterpret_cast<const float2*>(w.ws + w.hvf),
                                                            reinterpret_cast<const float2*>(w.ws + w.phf));
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_window_clear(Sim* s, int column) {
  pic_status st = launch_window_flush(s);   // never two pending columns
  if (st != PIC_OK) return st;
  const pic_config& c = s->cfg;
  WindowState& w = s->win;
  const size_t G = s->grid_elems();
  double2* colv = reinterpret_cast<double2*>(w.ws + w.colv);
  double2* hv = reinterpret_cast<double2*>(w.ws + w.hv);
  double2* ph = reinterpret_cast<double2*>(w.ws + w.ph);
  const int n_take = 2 * c.Nm * c.Nr;
  if (c.precision == PIC_FP64)
    k_win_col_take<double2><<<(n_take + kWinThreads - 1) / kWinThreads, kWinThreads, 0, s->stream>>>(
        s->at<double2>(s->lay.E), G, c.Nm, c.Nr, c.Nz, column, colv,
        eb_dw_active(s) ? s->at<float4>(s->lay.ebdw) : nullptr);
  else
    k_win_col_take<float2><<<(n_take + kWinThreads - 1) / kWinThreads, kWinThreads, 0, s->stream>>>(
        s->at<float2>(s->lay.E), G, c.Nm, c.Nr, c.Nz, column, colv, nullptr);
  PIC_LAUNCHED(s);
  const int n_out = 6 * c.Nm * c.Nr;
  const int hb = (n_out * 32 + kWinThreads - 1) / kWinThreads;
  const int pb = (c.Nz + kWinThreads - 1) / kWinThreads;
  k_win_col_hankel<<<hb + pb, kWinThreads, 0, s->stream>>>(s->at<double>(s->lay.mfwd), c.Nm, c.Nr, colv, hv, hb, ph,
                                                           c.Nz, column, reinterpret_cast<float2*>(w.ws + w.hvf),
                                                           reinterpret_cast<float2*>(w.ws + w.phf));
  PIC_LAUNCHED(s);
  w.pending = 1;
  return PIC_OK;
}

}  // namespace pic
