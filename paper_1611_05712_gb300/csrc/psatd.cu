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
// One thread per spectral cell; every grid is read once and written once.
#include "pic_internal.cuh"

namespace pic {
namespace {

struct Z {
  double re, im;
};
__device__ __forceinline__ Z zld(const double2* p, size_t i) { double2 v = p[i]; return {v.x, v.y}; }
__device__ __forceinline__ void zst(double2* p, size_t i, Z v) { p[i] = make_double2(v.re, v.im); }
__device__ __forceinline__ Z zadd(Z a, Z b) { return {a.re + b.re, a.im + b.im}; }
__device__ __forceinline__ Z zsub(Z a, Z b) { return {a.re - b.re, a.im - b.im}; }
__device__ __forceinline__ Z zscale(double s, Z a) { return {s * a.re, s * a.im}; }
__device__ __forceinline__ Z zi(double s, Z a) { return {-s * a.im, s * a.re}; }   // i s a

__global__ void __launch_bounds__(256) k_psatd_f64(double2* __restrict__ Eh, double2* __restrict__ Bh,
                                                   const double2* __restrict__ src,
                                                   double2* __restrict__ rho_prev,
                                                   const double* __restrict__ coef,
                                                   const double* __restrict__ kperp,
                                                   const double* __restrict__ kzmod,
                                                   const double* __restrict__ tz,
                                                   const double* __restrict__ tr, int Nz, size_t G,
                                                   double dt, int filter) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = idx % Nz;
    const size_t mn = idx / Nz;
    const double Kp = kperp[mn], Kz = kzmod[kz];
    const double T = filter ? tz[kz] * tr[mn] : 1.0;
    Z rn = zscale(T, zld(src, idx));
    Z Jp = zscale(T, zld(src, G + idx));
    Z Jm = zscale(T, zld(src, 2 * G + idx));
    Z Jz = zscale(T, zld(src, 3 * G + idx));
    const Z rp = zld(rho_prev, idx);
    const double C = coef[idx], SK = coef[G + idx], omc = coef[2 * G + idx];
    const double an = coef[3 * G + idx], ap = coef[4 * G + idx], iK2 = coef[5 * G + idx];
    // current correction
    Z divJ = zadd(zscale(Kp, zsub(Jp, Jm)), zi(Kz, Jz));
    Z Gc = zscale(iK2, zadd(zscale(1.0 / dt, zsub(rn, rp)), divJ));
    Jp = zadd(Jp, zscale(-0.5 * Kp, Gc));
    Jm = zadd(Jm, zscale(0.5 * Kp, Gc));
    Jz = zadd(Jz, zi(Kz, Gc));
    const Z Ep = zld(Eh, idx), Em = zld(Eh, G + idx), Ez = zld(Eh, 2 * G + idx);
    const Z Bp = zld(Bh, idx), Bm = zld(Bh, G + idx), Bz = zld(Bh, 2 * G + idx);
    // curls
    const Z cBp = zsub(zscale(Kz, Bp), zi(0.5 * Kp, Bz));
    const Z cBm = zsub(zscale(-Kz, Bm), zi(0.5 * Kp, Bz));
    const Z cBz = zi(Kp, zadd(Bp, Bm));
    const Z cEp = zsub(zscale(Kz, Ep), zi(0.5 * Kp, Ez));
    const Z cEm = zsub(zscale(-Kz, Em), zi(0.5 * Kp, Ez));
    const Z cEz = zi(Kp, zadd(Ep, Em));
    const Z cJp = zsub(zscale(Kz, Jp), zi(0.5 * Kp, Jz));
    const Z cJm = zsub(zscale(-Kz, Jm), zi(0.5 * Kp, Jz));
    const Z cJz = zi(Kp, zadd(Jp, Jm));
    const Z X = zscale(1.0 / kEps0, zadd(zscale(an, rn), zscale(ap, rp)));
    const double cSK = kC * SK, jS = SK / (kEps0 * kC), bS = SK / kC, jB = kMu0 * omc;
    Z nEp = zadd(zadd(zscale(C, Ep), zscale(cSK, cBp)), zadd(zscale(-jS, Jp), zscale(-0.5 * Kp, X)));
    Z nEm = zadd(zadd(zscale(C, Em), zscale(cSK, cBm)), zadd(zscale(-jS, Jm), zscale(0.5 * Kp, X)));
    Z nEz = zadd(zadd(zscale(C, Ez), zscale(cSK, cBz)), zadd(zscale(-jS, Jz), zi(Kz, X)));
    Z nBp = zadd(zadd(zscale(C, Bp), zscale(-bS, cEp)), zscale(jB, cJp));
    Z nBm = zadd(zadd(zscale(C, Bm), zscale(-bS, cEm)), zscale(jB, cJm));
    Z nBz = zadd(zadd(zscale(C, Bz), zscale(-bS, cEz)), zscale(jB, cJz));
    zst(Eh, idx, nEp); zst(Eh, G + idx, nEm); zst(Eh, 2 * G + idx, nEz);
    zst(Bh, idx, nBp); zst(Bh, G + idx, nBm); zst(Bh, 2 * G + idx, nBz);
    zst(rho_prev, idx, rn);
  }
}

// Space-charge field of a beam moving along +z (initial condition): relativistic
// Poisson solve phi = rho/(eps0 (K_perp^2 + K_z^2/gamma^2)),
// E += (K_perp phi/2, -K_perp phi/2, -i K_z phi/gamma^2), B += curl(0, 0, beta phi/c).
__global__ void k_beam_fields(double2* __restrict__ Eh, double2* __restrict__ Bh,
                              const double2* __restrict__ rho, const double* __restrict__ kperp,
                              const double* __restrict__ kzmod, const double* __restrict__ tz,
                              const double* __restrict__ tr, int Nz, size_t G, double gamma,
                              int filter) {
  const double ig2 = 1.0 / (gamma * gamma);
  const double beta = sqrt(1.0 - ig2);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int kz = idx % Nz;
    const size_t mn = idx / Nz;
    const double Kp = kperp[mn], Kz = kzmod[kz];
    const double T = filter ? tz[kz] * tr[mn] : 1.0;
    const Z r = zscale(T, zld(rho, idx));
    const Z phi = zscale(1.0 / (kEps0 * (Kp * Kp + Kz * Kz * ig2)), r);
    const Z A = zscale(beta / kC, phi);
    zst(Eh, idx, zadd(zld(Eh, idx), zscale(0.5 * Kp, phi)));
    zst(Eh, G + idx, zadd(zld(Eh, G + idx), zscale(-0.5 * Kp, phi)));
    zst(Eh, 2 * G + idx, zadd(zld(Eh, 2 * G + idx), zi(-Kz * ig2, phi)));
    zst(Bh, idx, zadd(zld(Bh, idx), zi(-0.5 * Kp, A)));
    zst(Bh, G + idx, zadd(zld(Bh, G + idx), zi(-0.5 * Kp, A)));
  }
}

// dst[idx] = T * src[idx] (T = filter factor, or 1 when the filter is off)
__global__ void k_filter_copy(double2* __restrict__ dst, const double2* __restrict__ src,
                              const double* __restrict__ tz, const double* __restrict__ tr, int Nz,
                              size_t G, int filter) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < G;
       idx += (size_t)gridDim.x * blockDim.x) {
    const double T = filter ? tz[idx % Nz] * tr[idx / Nz] : 1.0;
    double2 v = src[idx];
    dst[idx] = make_double2(T * v.x, T * v.y);
  }
}

__global__ void k_scale_copy(double2* __restrict__ dst, const double2* __restrict__ src, double a,
                             size_t n) {
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < n;
       idx += (size_t)gridDim.x * blockDim.x) {
    double2 v = src[idx];
    dst[idx] = make_double2(a * v.x, a * v.y);
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
  k_psatd_f64<<<grid_for(G), 256, 0, s->stream>>>(
      s->at<double2>(s->lay.Eh), s->at<double2>(s->lay.Bh), s->at<double2>(s->lay.srch),
      s->at<double2>(s->lay.rho_prev_h), s->at<double>(s->lay.coef), s->at<double>(s->lay.kperp),
      s->at<double>(s->lay.kzmod), s->at<double>(s->lay.tz), s->at<double>(s->lay.tr), c.Nz, G, c.dt,
      c.filter);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_beam_fields(Sim* s, const void* rho_h, double gamma) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  k_beam_fields<<<grid_for(G), 256, 0, s->stream>>>(
      s->at<double2>(s->lay.Eh), s->at<double2>(s->lay.Bh), (const double2*)rho_h,
      s->at<double>(s->lay.kperp), s->at<double>(s->lay.kzmod), s->at<double>(s->lay.tz),
      s->at<double>(s->lay.tr), c.Nz, G, gamma, c.filter);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_scale_copy(Sim* s, void* dst, const void* src, double a, size_t n_cplx) {
  k_scale_copy<<<grid_for(n_cplx), 256, 0, s->stream>>>((double2*)dst, (const double2*)src, a, n_cplx);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

pic_status launch_filter_copy(Sim* s, void* dst, const void* src) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  k_filter_copy<<<grid_for(G), 256, 0, s->stream>>>((double2*)dst, (const double2*)src,
                                                    s->at<double>(s->lay.tz),
                                                    s->at<double>(s->lay.tr), c.Nz, G, c.filter);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
