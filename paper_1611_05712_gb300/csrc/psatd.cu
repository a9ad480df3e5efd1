// PSATD field update (a7) per spectral cell (m, n, k_z), SI form of Eq. psatd-eqE /
// psatd-eqB with the quasi-cylindrical operators of Eq. qcyl-ops and k_z -> [k_z]_p
// inside K, C and S (section "Finite order pseudo-spectral solvers"):
//   1. filter rho^{n+1}, J by T = cos^2(k_z dz/2) cos^2(k_perp dr/2)        (when on)
//   2. G = [(rho^{n+1}-rho^n)/dt + div J]/K^2 ; J += grad G      (global current correction)
//   3. E' = C E + c (S/K) curl B - (S/K)/(eps0 c) J + grad(a_n rho^{n+1} + a_p rho^n)/eps0
//      B' = C B - (S/K)/c curl E + mu0 (1-C)/K^2 curl J
//   4. rho^n <- rho^{n+1}
// grad X = (-K_perp X/2, K_perp X/2, i K_z X),
// curl V = (K_z V+ - i K_perp Vz/2, -K_z V- - i K_perp Vz/2, i K_perp (V+ + V-)),
// div V = K_perp (V+ - V-) + i K_z Vz.
// The float64 update never forms the corrected current J + grad G: in E' it enters as
// -(S/K)/(eps0 c) J - grad Y with Y = (S/K)/(eps0 c) G - (a_n rho^{n+1} + a_p rho^n)/eps0,
// and in B' only through its curl, which is curl J (curl grad = 0 for these operators: K_z
// (-K_perp G/2) - i (K_perp/2) (i K_z G) = 0, and so on), so B' = C B + curl W with W = mu0
// (1-C)/K^2 J - (S/K)/c E, one curl instead of two: fewer float64 operations, which bound the
// FP64 form's update.  The float update (bound by memory) keeps the steps written out.
// One thread per spectral cell; every grid is read once and written once.  R = double in
// the FP64 form, float (with float coefficient tables) in the mixed form.
#include "pic_internal.cuh"

namespace pic {
namespace {

template <typename R> struct V2;
template <> struct V2<double> { using T = double2; };
template <> struct V2<float> { using T = float2; };

template <typename R> struct Z {
  R re, im;
};
template <typename R> __device__ __forceinline__ Z<R> zld(const typename V2<R>::T* p, size_t i) {
  const typename V2<R>::T v = p[i];
  return {v.x, v.y};
}
template <typename R> __device__ __forceinline__ void zst(typename V2<R>::T* p, size_t i, Z<R> v) {
  typename V2<R>::T o;
  o.x = v.re;
  o.y = v.im;
  p[i] = o;
}
template <typename R> __device__ __forceinline__ Z<R> zadd(Z<R> a, Z<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ Z<R> zsub(Z<R> a, Z<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ Z<R> zscale(R s, Z<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __device__ __forceinline__ Z<R> zi(R s, Z<R> a) { return {-s * a.im, s * a.re}; }  // i s a

// v -= h p: subtraction of a departed window column's transform (moving window); the
// mixed form reads h and p rounded to float.
template <typename R, typename T2>
__device__ __forceinline__ void col_sub(Z<R>& v, T2 h, T2 p) {
  v.re -= h.x * p.x - h.y * p.y;
  v.im -= h.x * p.y + h.y * p.x;
}

// PEND: a moving-window column removal is pending and applied to E^, B^ as they are loaded.
template <typename R, bool PEND>
__global__ void __launch_bounds__(256) k_psatd(typename V2<R>::T* __restrict__ Eh, typename V2<R>::T* __restrict__ Bh,
                                               const typename V2<R>::T* __restrict__ src,
                                               typename V2<R>::T* __restrict__ rho_prev,
                                               const R* __restrict__ coef, const R* __restrict__ kperp,
                                               const R* __restrict__ kzmod, const R* __restrict__ tz,
                                               const R* __restrict__ tr, int Nz, size_t G, double dt,
                                               int filter, const typename V2<R>::T* __restrict__ colh,
                                               const typename V2<R>::T* __restrict__ colph) {
  const R kc = (R)kC, ieps0 = (R)(1.0 / kEps0), idt = (R)(1.0 / dt);
  const R jS_f = (R)(1.0 / (kEps0 * kC)), bS_f = (R)(1.0 / kC), mu0 = (R)kMu0;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = idx % Nz;
    const size_t mn = idx / Nz;
    const R Kp = kperp[mn], Kz = kzmod[kz];
    const R T = filter ? tz[kz] * tr[mn] : (R)1;
    Z<R> rn = zscale(T, zld<R>(src, idx));
    Z<R> Jp = zscale(T, zld<R>(src, G + idx));
    Z<R> Jm = zscale(T, zld<R>(src, 2 * G + idx));
    Z<R> Jz = zscale(T, zld<R>(src, 3 * G + idx));
    const Z<R> rp = zld<R>(rho_prev, idx);
    const R C = coef[idx], SK = coef[G + idx], omc = coef[2 * G + idx];
    const R an = coef[3 * G + idx], ap = coef[4 * G + idx], iK2 = coef[5 * G + idx];
    const R h = (R)0.5;
    if constexpr (sizeof(R) == 8) {   // float64: the folded update (fewer float64 operations)
      // current correction: G only (the corrected current is never formed, see below)
      const Z<R> divJ = zadd(zscale(Kp, zsub(Jp, Jm)), zi(Kz, Jz));
      const Z<R> Gc = zscale(iK2, zadd(zscale(idt, zsub(rn, rp)), divJ));
      Z<R> Ep = zld<R>(Eh, idx), Em = zld<R>(Eh, G + idx), Ez = zld<R>(Eh, 2 * G + idx);
      Z<R> Bp = zld<R>(Bh, idx), Bm = zld<R>(Bh, G + idx), Bz = zld<R>(Bh, 2 * G + idx);
      if (PEND) {   // pending removal of the moving window's departed column: F^ -= h[row] p[k]
        const typename V2<R>::T p = colph[kz];
        const size_t MN = G / Nz;
        col_sub(Ep, colh[mn], p); col_sub(Em, colh[MN + mn], p); col_sub(Ez, colh[2 * MN + mn], p);
        col_sub(Bp, colh[3 * MN + mn], p); col_sub(Bm, colh[4 * MN + mn], p); col_sub(Bz, colh[5 * MN + mn], p);
      }
      const R hK = h * Kp;
      const Z<R> cBp = zsub(zscale(Kz, Bp), zi(hK, Bz));
      const Z<R> cBm = zsub(zscale(-Kz, Bm), zi(hK, Bz));
      const Z<R> cBz = zi(Kp, zadd(Bp, Bm));
      const Z<R> X = zscale(ieps0, zadd(zscale(an, rn), zscale(ap, rp)));
      const R cSK = kc * SK, jS = SK * jS_f, bS = SK * bS_f, jB = mu0 * omc;
      // E' = C E + c (S/K) curl B - (S/K)/(eps0 c) J - grad Y,  Y = (S/K)/(eps0 c) G - X
      const Z<R> Y = zsub(zscale(jS, Gc), X);
      const Z<R> nEp = zadd(zadd(zscale(C, Ep), zscale(cSK, cBp)), zadd(zscale(-jS, Jp), zscale(hK, Y)));
      const Z<R> nEm = zadd(zadd(zscale(C, Em), zscale(cSK, cBm)), zsub(zscale(-jS, Jm), zscale(hK, Y)));
      const Z<R> nEz = zadd(zadd(zscale(C, Ez), zscale(cSK, cBz)), zsub(zscale(-jS, Jz), zi(Kz, Y)));
      // B' = C B + curl W,  W = mu0 (1-C)/K^2 J - (S/K)/c E  (old E; curl grad G = 0)
      const Z<R> Wp = zsub(zscale(jB, Jp), zscale(bS, Ep));
      const Z<R> Wm = zsub(zscale(jB, Jm), zscale(bS, Em));
      const Z<R> Wz = zsub(zscale(jB, Jz), zscale(bS, Ez));
      const Z<R> nBp = zadd(zscale(C, Bp), zsub(zscale(Kz, Wp), zi(hK, Wz)));
      const Z<R> nBm = zadd(zscale(C, Bm), zsub(zscale(-Kz, Wm), zi(hK, Wz)));
      const Z<R> nBz = zadd(zscale(C, Bz), zi(Kp, zadd(Wp, Wm)));
      zst<R>(Eh, idx, nEp); zst<R>(Eh, G + idx, nEm); zst<R>(Eh, 2 * G + idx, nEz);
      zst<R>(Bh, idx, nBp); zst<R>(Bh, G + idx, nBm); zst<R>(Bh, 2 * G + idx, nBz);
      zst<R>(rho_prev, idx, rn);
    } else {   // float: written out (the folded form ran 7 % slower in this memory-bound kernel)
      // current correction
      const Z<R> divJ = zadd(zscale(Kp, zsub(Jp, Jm)), zi(Kz, Jz));
      const Z<R> Gc = zscale(iK2, zadd(zscale(idt, zsub(rn, rp)), divJ));
      Jp = zadd(Jp, zscale(-h * Kp, Gc));
      Jm = zadd(Jm, zscale(h * Kp, Gc));
      Jz = zadd(Jz, zi(Kz, Gc));
      Z<R> Ep = zld<R>(Eh, idx), Em = zld<R>(Eh, G + idx), Ez = zld<R>(Eh, 2 * G + idx);
      Z<R> Bp = zld<R>(Bh, idx), Bm = zld<R>(Bh, G + idx), Bz = zld<R>(Bh, 2 * G + idx);
      if (PEND) {   // pending removal of the moving window's departed column: F^ -= h[row] p[k]
        const typename V2<R>::T p = colph[kz];
        const size_t MN = G / Nz;
        col_sub(Ep, colh[mn], p); col_sub(Em, colh[MN + mn], p); col_sub(Ez, colh[2 * MN + mn], p);
        col_sub(Bp, colh[3 * MN + mn], p); col_sub(Bm, colh[4 * MN + mn], p); col_sub(Bz, colh[5 * MN + mn], p);
      }
      // curls
      const Z<R> cBp = zsub(zscale(Kz, Bp), zi(h * Kp, Bz));
      const Z<R> cBm = zsub(zscale(-Kz, Bm), zi(h * Kp, Bz));
      const Z<R> cBz = zi(Kp, zadd(Bp, Bm));
      const Z<R> cEp = zsub(zscale(Kz, Ep), zi(h * Kp, Ez));
      const Z<R> cEm = zsub(zscale(-Kz, Em), zi(h * Kp, Ez));
      const Z<R> cEz = zi(Kp, zadd(Ep, Em));
      const Z<R> cJp = zsub(zscale(Kz, Jp), zi(h * Kp, Jz));
      const Z<R> cJm = zsub(zscale(-Kz, Jm), zi(h * Kp, Jz));
      const Z<R> cJz = zi(Kp, zadd(Jp, Jm));
      const Z<R> X = zscale(ieps0, zadd(zscale(an, rn), zscale(ap, rp)));
      const R cSK = kc * SK, jS = SK * jS_f, bS = SK * bS_f, jB = mu0 * omc;
      const Z<R> nEp = zadd(zadd(zscale(C, Ep), zscale(cSK, cBp)), zadd(zscale(-jS, Jp), zscale(-h * Kp, X)));
      const Z<R> nEm = zadd(zadd(zscale(C, Em), zscale(cSK, cBm)), zadd(zscale(-jS, Jm), zscale(h * Kp, X)));
      const Z<R> nEz = zadd(zadd(zscale(C, Ez), zscale(cSK, cBz)), zadd(zscale(-jS, Jz), zi(Kz, X)));
      const Z<R> nBp = zadd(zadd(zscale(C, Bp), zscale(-bS, cEp)), zscale(jB, cJp));
      const Z<R> nBm = zadd(zadd(zscale(C, Bm), zscale(-bS, cEm)), zscale(jB, cJm));
      const Z<R> nBz = zadd(zadd(zscale(C, Bz), zscale(-bS, cEz)), zscale(jB, cJz));
      zst<R>(Eh, idx, nEp); zst<R>(Eh, G + idx, nEm); zst<R>(Eh, 2 * G + idx, nEz);
      zst<R>(Bh, idx, nBp); zst<R>(Bh, G + idx, nBm); zst<R>(Bh, 2 * G + idx, nBz);
      zst<R>(rho_prev, idx, rn);
    }
  }
}

// Space-charge field of a beam moving along +z (initial condition): relativistic
// Poisson solve phi = rho/(eps0 (K_perp^2 + K_z^2/gamma^2)),
// E += (K_perp phi/2, -K_perp phi/2, -i K_z phi/gamma^2), B += curl(0, 0, beta phi/c).
// Always evaluated in float64; the mixed form reads and writes float grids.
template <typename R>
__global__ void k_beam_fields(typename V2<R>::T* __restrict__ Eh, typename V2<R>::T* __restrict__ Bh,
                              const typename V2<R>::T* __restrict__ rho, const double* __restrict__ kperp,
                              const double* __restrict__ kzmod, const double* __restrict__ tz,
                              const double* __restrict__ tr, int Nz, size_t G, double gamma, int filter) {
  const double ig2 = 1.0 / (gamma * gamma);
  const double beta = sqrt(1.0 - ig2);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = idx % Nz;
    const size_t mn = idx / Nz;
    const double Kp = kperp[mn], Kz = kzmod[kz];
    const double T = filter ? tz[kz] * tr[mn] : 1.0;
    const Z<R> r0 = zld<R>(rho, idx);
    const Z<double> r = {T * (double)r0.re, T * (double)r0.im};
    const Z<double> phi = zscale(1.0 / (kEps0 * (Kp * Kp + Kz * Kz * ig2)), r);
    const Z<double> A = zscale(beta / kC, phi);
    const Z<double> add[5] = {zscale(0.5 * Kp, phi), zscale(-0.5 * Kp, phi), zi(-Kz * ig2, phi),
                              zi(-0.5 * Kp, A), zi(-0.5 * Kp, A)};
    typename V2<R>::T* dst[5] = {Eh, Eh, Eh, Bh, Bh};
    const size_t off[5] = {idx, G + idx, 2 * G + idx, idx, G + idx};
    for (int k = 0; k < 5; ++k) {
      const Z<R> v = zld<R>(dst[k], off[k]);
      zst<R>(dst[k], off[k], Z<R>{(R)((double)v.re + add[k].re), (R)((double)v.im + add[k].im)});
    }
  }
}

// dst[idx] = T * src[idx] (T = filter factor, or 1 when the filter is off)
template <typename R>
__global__ void k_filter_copy(typename V2<R>::T* __restrict__ dst, const typename V2<R>::T* __restrict__ src,
                              const double* __restrict__ tz, const double* __restrict__ tr, int Nz,
                              size_t G, int filter) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const double T = filter ? tz[idx % Nz] * tr[idx / Nz] : 1.0;
    const Z<R> v = zld<R>(src, idx);
    zst<R>(dst, idx, Z<R>{(R)(T * v.re), (R)(T * v.im)});
  }
}

template <typename R>
__global__ void k_scale_copy(typename V2<R>::T* __restrict__ dst, const typename V2<R>::T* __restrict__ src,
                             double a, size_t n) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    const Z<R> v = zld<R>(src, idx);
    zst<R>(dst, idx, Z<R>{(R)(a * v.re), (R)(a * v.im)});
  }
}

inline int grid_for(size_t n) {
  size_t b = (n + 255) / 256;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

}  // namespace

pic_status launch_psatd(Sim* s) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  const bool pend = s->win.pending != 0;
  s->win.pending = 0;
  const char* wb = s->win.ws;
  if (c.precision == PIC_FP64) {
    auto* k = pend ? k_psatd<double, true> : k_psatd<double, false>;
    k<<<grid_for(G), 256, 0, s->stream>>>(
        s->at<double2>(s->lay.Eh), s->at<double2>(s->lay.Bh), s->at<double2>(s->lay.srch),
        s->at<double2>(s->lay.rho_prev_h), s->at<double>(s->lay.coef), s->at<double>(s->lay.kperp),
        s->at<double>(s->lay.kzmod), s->at<double>(s->lay.tz), s->at<double>(s->lay.tr), c.Nz, G, c.dt,
        c.filter, pend ? reinterpret_cast<const double2*>(wb + s->win.hv) : nullptr,
        pend ? reinterpret_cast<const double2*>(wb + s->win.ph) : nullptr);
  } else {
    auto* k = pend ? k_psatd<float, true> : k_psatd<float, false>;
    k<<<grid_for(G), 256, 0, s->stream>>>(
        s->at<float2>(s->lay.Eh), s->at<float2>(s->lay.Bh), s->at<float2>(s->lay.srch),
        s->at<float2>(s->lay.rho_prev_h), s->at<float>(s->lay.coef_f), s->at<float>(s->lay.kperp_f),
        s->at<float>(s->lay.kzmod_f), s->at<float>(s->lay.tz_f), s->at<float>(s->lay.tr_f), c.Nz, G, c.dt,
        c.filter, pend ? reinterpret_cast<const float2*>(wb + s->win.hvf) : nullptr,
        pend ? reinterpret_cast<const float2*>(wb + s->win.phf) : nullptr);
  }
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_beam_fields(Sim* s, const void* rho_h, double gamma) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  if (c.precision == PIC_FP64)
    k_beam_fields<double><<<grid_for(G), 256, 0, s->stream>>>(
        s->at<double2>(s->lay.Eh), s->at<double2>(s->lay.Bh), (const double2*)rho_h, s->at<double>(s->lay.kperp),
        s->at<double>(s->lay.kzmod), s->at<double>(s->lay.tz), s->at<double>(s->lay.tr), c.Nz, G, gamma, c.filter);
  else
    k_beam_fields<float><<<grid_for(G), 256, 0, s->stream>>>(
        s->at<float2>(s->lay.Eh), s->at<float2>(s->lay.Bh), (const float2*)rho_h, s->at<double>(s->lay.kperp),
        s->at<double>(s->lay.kzmod), s->at<double>(s->lay.tz), s->at<double>(s->lay.tr), c.Nz, G, gamma, c.filter);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_scale_copy(Sim* s, void* dst, const void* src, double a, size_t n_cplx) {
  if (s->cfg.precision == PIC_FP64)
    k_scale_copy<double><<<grid_for(n_cplx), 256, 0, s->stream>>>((double2*)dst, (const double2*)src, a, n_cplx);
  else
    k_scale_copy<float><<<grid_for(n_cplx), 256, 0, s->stream>>>((float2*)dst, (const float2*)src, a, n_cplx);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_filter_copy(Sim* s, void* dst, const void* src) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  if (c.precision == PIC_FP64)
    k_filter_copy<double><<<grid_for(G), 256, 0, s->stream>>>((double2*)dst, (const double2*)src,
                                                              s->at<double>(s->lay.tz), s->at<double>(s->lay.tr),
                                                              c.Nz, G, c.filter);
  else
    k_filter_copy<float><<<grid_for(G), 256, 0, s->stream>>>((float2*)dst, (const float2*)src,
                                                             s->at<double>(s->lay.tz), s->at<double>(s->lay.tr),
                                                             c.Nz, G, c.filter);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
