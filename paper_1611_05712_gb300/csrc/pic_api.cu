// C ABI of libpsatd_rz.so (declared in include/psatd_rz.h): configuration checks,
// workspace layout, and the order of the stages of one quasi-cylindrical PSATD PIC cycle
// (section "Finite order pseudo-spectral solvers" of arXiv:1611.05712).
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <utility>
#include <vector>

#include "pic_internal.cuh"

namespace pic {

static thread_local std::string g_last_error;

void set_error(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
}

pic_status cuda_status(cudaError_t e, const char* what) {
  set_error("%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
  return PIC_ERR_CUDA;
}

bool plan_radix(int N, int32_t* radix, int32_t* n_pass);
size_t diag_acc_doubles();
pic_status launch_filter_copy(Sim* s, void* dst, const void* src);
pic_status launch_scale_copy(Sim* s, void* dst, const void* src, double a, size_t n_cplx);

namespace {

pic_status validate(const pic_config* c, int32_t* radix, int32_t* n_pass) {
  if (!c) { set_error("config is NULL"); return PIC_ERR_ARG; }
  if (c->precision != PIC_FP64 && c->precision != PIC_MIXED_TF32X3 && c->precision != PIC_MIXED_BF16X6) {
    set_error("precision %d is not a pic_precision", c->precision);
    return PIC_ERR_ARG;
  }
  // power-of-two rows hold one row per FFT CTA in shared memory, other lengths two (the
  // float64 form's rows of other lengths therefore stop at 4096)
  const bool pow2 = (c->Nz & (c->Nz - 1)) == 0;
  const int max_nz = c->precision == PIC_FP64 && !pow2 ? 4096 : 8192;
  if (c->Nz < 8 || c->Nz > max_nz) {
    set_error("Nz=%d must be in [8, %d]%s", c->Nz, max_nz, max_nz == 4096 ? " (float64 rows of a length that is not a power of two)" : "");
    return PIC_ERR_ARG;
  }
  if (!plan_radix(c->Nz, radix, n_pass)) {
    *n_pass = 0;
    if (bluestein_length(c->Nz, c->precision) == 0) {
      set_error("Nz=%d is not 7-smooth: Bluestein lengths reach Nz <= %d", c->Nz, max_nz / 2);
      return PIC_ERR_ARG;
    }
  }
  if (c->Nr < 4 || c->Nr > kMaxNr) { set_error("Nr=%d must be in [4, %d]", c->Nr, kMaxNr); return PIC_ERR_ARG; }
  if (c->Nm < 1 || c->Nm > kMaxModes) { set_error("Nm=%d must be in [1, %d]", c->Nm, kMaxModes); return PIC_ERR_ARG; }
  if (c->order_p != 0 && (c->order_p < 2 || c->order_p > 512 || (c->order_p & 1))) {
    set_error("order_p=%d must be 0 (infinite) or even in [2, 512]", c->order_p);
    return PIC_ERR_ARG;
  }
  if (!(c->dz > 0) || !(c->dr > 0) || !(c->dt > 0)) { set_error("dz, dr, dt must be > 0"); return PIC_ERR_ARG; }
  if (c->np_capacity < 0 || c->np_capacity > INT32_MAX) {
    set_error("np_capacity=%lld out of range", (long long)c->np_capacity);
    return PIC_ERR_ARG;
  }
  if (!(c->mass > 0) || !(c->q == c->q)) { set_error("species charge/mass invalid"); return PIC_ERR_ARG; }
  return PIC_OK;
}

Layout make_layout(const pic_config& c) {
  Layout L{};
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const bool mixed = c.precision != PIC_FP64;
  const size_t cb = mixed ? 8 : 16;   // complex float64 or complex float
  const size_t G = (size_t)c.Nm * c.Nr * c.Nz;
  const size_t Nr2 = (size_t)c.Nr * c.Nr;
  const size_t cap = (size_t)std::max<int64_t>(c.np_capacity, 1);
  const size_t ncell = (size_t)c.Nz * c.Nr;
  L.E = take(6 * G * cb);   // E then B, adjacent
  L.B = L.E + 3 * G * cb;
  L.Eh = take(6 * G * cb);  // Eh then Bh, adjacent
  L.Bh = L.Eh + 3 * G * cb;
  L.dep = take(4 * G * cb);
  L.srch = take(4 * G * cb);
  L.tmp = take(6 * G * cb);
  L.rho_prev_h = take(G * cb);
  L.rho_ion = take(G * cb);
  L.kperp = take((size_t)c.Nm * c.Nr * 8);
  L.binv = take((size_t)c.Nm * 3 * Nr2 * 8);
  L.mfwd = take((size_t)c.Nm * 3 * Nr2 * 8);
  L.svd_w = take((size_t)c.Nm * 3 * Nr2 * 8);
  L.svd_v = take((size_t)c.Nm * 3 * Nr2 * 8);
  L.svd_d = take((size_t)c.Nm * 3 * c.Nr * 8);
  L.kzmod = take((size_t)c.Nz * 8);
  L.tz = take((size_t)c.Nz * 8);
  L.tr = take((size_t)c.Nm * c.Nr * 8);
  L.coef = take(6 * G * 8);
  L.twp = take((size_t)c.Nz * 16);
  if (c.precision == PIC_FP64) L.twp_dw = take((size_t)c.Nz * 16);
  if (c.precision == PIC_FP64 && fft_is_pow2(c.Nz)) L.ebdw = take(6 * G * 16);
  const int M = bluestein_length(c.Nz, c.precision);
  if (M > 0) {
    L.twm = take((size_t)M * 16);
    L.chirp = take((size_t)c.Nz * 16);
    L.bspec = take((size_t)M * 16);
    if (c.precision != PIC_FP64) {
      L.twm_f = take((size_t)M * 8);
      L.chirp_f = take((size_t)c.Nz * 8);
      L.bspec_f = take((size_t)M * 8);
    }
  }
  if (f64s_supported(c)) {
    const size_t pitch = (size_t)split_pitch_b16(c.Nr), Nc = 2 * (size_t)c.Nz, nmat = 6 * (size_t)c.Nm;
    L.f64s_mat = take(nmat * kF64sSlices * c.Nr * pitch * 2);
    L.f64s_rowexp = take(nmat * c.Nr * 4);
    L.f64s_panel = take(nmat * kF64sSlices * Nc * pitch * 2);
    L.f64s_colexp = take(nmat * Nc * 4 + nmat * Nc * 8);   // exponents, then the column maxima
  }
  if (mixed) {
    for (int b = 0; b < 2; ++b)
      for (int k = 0; k < kPfCount; ++k) L.pf[b][k] = take(cap * 4);
    L.stage64 = take(7 * cap * 8);
    L.ebt = take(6 * G * 8);
    L.coef_f = take(6 * G * 4);
    L.kperp_f = take((size_t)c.Nm * c.Nr * 4);
    L.kzmod_f = take((size_t)c.Nz * 4);
    L.tz_f = take((size_t)c.Nz * 4);
    L.tr_f = take((size_t)c.Nm * c.Nr * 4);
    L.twp_f = take((size_t)c.Nz * 8);
    if (c.precision == PIC_MIXED_BF16X6) {
      // three BF16 planes per matrix, rows padded to 16 bytes
      const size_t plane = (size_t)c.Nm * 3 * c.Nr * split_pitch_b16(c.Nr) * 2;
      L.mfwd_hi = take(3 * plane);
      L.binv_hi = take(3 * plane);
    } else {
      L.mfwd_hi = take((size_t)c.Nm * 3 * c.Nr * split_pitch(c.Nr) * 4);
      L.mfwd_lo = take((size_t)c.Nm * 3 * c.Nr * split_pitch(c.Nr) * 4);
      L.binv_hi = take((size_t)c.Nm * 3 * c.Nr * split_pitch(c.Nr) * 4);
      L.binv_lo = take((size_t)c.Nm * 3 * c.Nr * split_pitch(c.Nr) * 4);
    }
  } else {
    for (int b = 0; b < 2; ++b) {
      for (int k = 0; k < 7; ++k) L.part[b][k] = take(cap * 8);
      L.pid[b] = take(cap * 4);
    }
  }
  L.keys = take(cap * 4);
  L.perm = take(cap * 4);
  L.perm_tmp = take(cap * 4);
  L.count = take((ncell + 66) * 4);   // cells plus 64 sub-bins of inactive particles (+1)
  L.start = take((ncell + 66) * 4);
  L.scan_blk = take(4 * 4096 * 4 + (ncell + 66) * 4);   // block totals, then the scatter cursor
  L.big_list = take(ncell * 4);
  L.big_count = take(256);
  L.diag_acc = take(diag_acc_doubles() * 8);
  L.err = take(256);
  L.total = off;
  return L;
}

struct BufView {
  size_t off, bytes;
};

bool buffer_view(const Sim* s, int32_t id, BufView* v) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems(), cb = s->cplx_bytes, Nr2 = (size_t)c.Nr * c.Nr;
  switch (id) {
    case PIC_BUF_E: *v = {s->lay.E, 3 * G * cb}; return true;
    case PIC_BUF_B: *v = {s->lay.B, 3 * G * cb}; return true;
    case PIC_BUF_EH: *v = {s->lay.Eh, 3 * G * cb}; return true;
    case PIC_BUF_BH: *v = {s->lay.Bh, 3 * G * cb}; return true;
    case PIC_BUF_DEP: *v = {s->lay.dep, 4 * G * cb}; return true;
    case PIC_BUF_SRC_H: *v = {s->lay.srch, 4 * G * cb}; return true;
    case PIC_BUF_RHO_PREV_H: *v = {s->lay.rho_prev_h, G * cb}; return true;
    case PIC_BUF_RHO_ION: *v = {s->lay.rho_ion, G * cb}; return true;
    case PIC_BUF_KPERP: *v = {s->lay.kperp, (size_t)c.Nm * c.Nr * 8}; return true;
    case PIC_BUF_HANKEL_INV: *v = {s->lay.binv, (size_t)c.Nm * 3 * Nr2 * 8}; return true;
    case PIC_BUF_HANKEL_FWD: *v = {s->lay.mfwd, (size_t)c.Nm * 3 * Nr2 * 8}; return true;
    case PIC_BUF_KZ_MOD: *v = {s->lay.kzmod, (size_t)c.Nz * 8}; return true;
    case PIC_BUF_KEYS: *v = {s->lay.keys, (size_t)s->np * 4}; return true;
    case PIC_BUF_PERM: *v = {s->lay.perm, (size_t)s->np * 4}; return true;
    default: return false;
  }
}

// forward z-FFT of the first n_comp components of dep into tmp, with
// J_+- = (J_r -+ i J_theta)/2 formed on load.
pic_status fft_forward(Sim* s, int n_comp) {
  RowCombine rc{};
  rc.n_out = n_comp;
  for (int k = 0; k < 6; ++k) { rc.srcA[k] = k; rc.srcB[k] = -1; rc.caRe[k] = 1.0; }
  if (n_comp == 4) {
    // out: rho, J_+ = (J_r - i J_th)/2, J_- = (J_r + i J_th)/2, J_z
    rc.srcA[1] = 1; rc.caRe[1] = 0.5; rc.srcB[1] = 2; rc.cbRe[1] = 0.0; rc.cbIm[1] = -0.5;
    rc.srcA[2] = 1; rc.caRe[2] = 0.5; rc.srcB[2] = 2; rc.cbRe[2] = 0.0; rc.cbIm[2] = 0.5;
    rc.srcA[3] = 3;
  }
  return launch_fft_rows(s, s->at<char>(s->lay.dep), s->at<char>(s->lay.tmp), rc, false);
}

// forward DHT of every (component, mode) of tmp into srch.
pic_status dht_forward(Sim* s, int n_comp) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  DhtBatch b{};
  const int slot_of[4] = {1, 2, 0, 1};   // rho: order m, J_+: m+1, J_-: m-1, J_z: m
  const size_t Nr2 = (size_t)c.Nr * c.Nr;
  for (int comp = 0; comp < n_comp; ++comp)
    for (int m = 0; m < c.Nm; ++m) {
      const size_t moff = ((size_t)m * 3 + slot_of[comp]) * Nr2;
      if (s->cfg.precision == PIC_FP64) b.A[b.n] = s->at<double>(s->lay.mfwd) + moff;
      b.mat[b.n] = (int16_t)(m * 3 + slot_of[comp]);   // the tensor maps select the matrix
      b.X[b.n] = s->at<char>(s->lay.tmp) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      b.Y[b.n] = s->at<char>(s->lay.srch) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      ++b.n;
    }
  return launch_dht(s, b);
}

// Forward transforms of the real-space fields into the spectral state: z-FFT of E, B with
// F_+- = (F_r -+ i F_theta)/2 formed on load, then the DHT of orders m+1, m-1, m into Eh, Bh.
pic_status fields_forward(Sim* s) {
  const pic_config& c = s->cfg;
  RowCombine rc{};
  rc.n_out = 6;
  for (int f = 0; f < 2; ++f) {
    const int o = 3 * f;
    rc.srcA[o + 0] = o; rc.caRe[o + 0] = 0.5; rc.srcB[o + 0] = o + 1; rc.cbIm[o + 0] = -0.5;
    rc.srcA[o + 1] = o; rc.caRe[o + 1] = 0.5; rc.srcB[o + 1] = o + 1; rc.cbIm[o + 1] = 0.5;
    rc.srcA[o + 2] = o + 2; rc.caRe[o + 2] = 1.0; rc.srcB[o + 2] = -1;
  }
  pic_status st = launch_fft_rows(s, s->at<char>(s->lay.E), s->at<char>(s->lay.tmp), rc, false);
  if (st != PIC_OK) return st;
  const size_t G = s->grid_elems();
  const size_t Nr2 = (size_t)c.Nr * c.Nr;
  const int slot_of[3] = {2, 0, 1};      // +: m+1, -: m-1, z: m
  DhtBatch b{};
  for (int comp = 0; comp < 6; ++comp)
    for (int m = 0; m < c.Nm; ++m) {
      const int slot = slot_of[comp % 3];
      if (c.precision == PIC_FP64) b.A[b.n] = s->at<double>(s->lay.mfwd) + ((size_t)m * 3 + slot) * Nr2;
      b.mat[b.n] = (int16_t)(m * 3 + slot);
      b.X[b.n] = s->at<char>(s->lay.tmp) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      b.Y[b.n] = s->at<char>(s->lay.Eh) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      ++b.n;
    }
  return launch_dht(s, b);
}

pic_status forward_transform(Sim* s, int n_comp) {
  pic_status st = fft_forward(s, n_comp);
  if (st != PIC_OK) return st;
  return dht_forward(s, n_comp);
}

// inverse DHT of Eh, Bh (+, -, z) per mode into tmp.
pic_status dht_inverse(Sim* s) {
  const pic_config& c = s->cfg;
  const size_t G = s->grid_elems();
  const size_t Nr2 = (size_t)c.Nr * c.Nr;
  const int slot_of[3] = {2, 0, 1};      // +: m+1, -: m-1, z: m
  DhtBatch b{};
  for (int comp = 0; comp < 6; ++comp)
    for (int m = 0; m < c.Nm; ++m) {
      const size_t moff = ((size_t)m * 3 + slot_of[comp % 3]) * Nr2;
      if (s->cfg.precision == PIC_FP64) b.A[b.n] = s->at<double>(s->lay.binv) + moff;
      b.mat[b.n] = (int16_t)(kMaxModes * 3 + m * 3 + slot_of[comp % 3]);
      b.X[b.n] = s->at<char>(s->lay.Eh) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      b.Y[b.n] = s->at<char>(s->lay.tmp) + ((size_t)comp * G + (size_t)m * c.Nr * c.Nz) * s->cplx_bytes;
      ++b.n;
    }
  return launch_dht(s, b);
}

// inverse z-FFT of tmp into E, B with E_r = E_+ + E_-, E_theta = i (E_+ - E_-) formed on load.
pic_status fft_inverse(Sim* s) {
  RowCombine rc{};
  rc.n_out = 6;
  for (int f = 0; f < 2; ++f) {
    const int o = 3 * f;
    rc.srcA[o + 0] = o; rc.caRe[o + 0] = 1.0; rc.srcB[o + 0] = o + 1; rc.cbRe[o + 0] = 1.0;
    rc.srcA[o + 1] = o; rc.caIm[o + 1] = 1.0; rc.srcB[o + 1] = o + 1; rc.cbIm[o + 1] = -1.0;
    rc.srcA[o + 2] = o + 2; rc.caRe[o + 2] = 1.0; rc.srcB[o + 2] = -1;
  }
  rc.out_dw = eb_dw_active(s) ? s->at<char>(s->lay.ebdw) : nullptr;
  return launch_fft_rows(s, s->at<char>(s->lay.tmp), s->at<char>(s->lay.E), rc, true);
}

pic_status inverse_transform(Sim* s) {
  pic_status st = dht_inverse(s);
  if (st != PIC_OK) return st;
  return fft_inverse(s);
}

pic_status deposit_rho_with_background(Sim* s) {
  const size_t G = s->grid_elems();
  PIC_CUDA(cudaMemcpyAsync(s->at<char>(s->lay.dep), s->at<char>(s->lay.rho_ion), G * s->cplx_bytes,
                           cudaMemcpyDeviceToDevice, s->stream));
  return launch_deposit(s, PIC_DEP_RHO, INT32_MIN, INT32_MAX, nullptr);
}

// Optional stage timing: when ev is non-null, ev[k] is recorded after stage k-1.
struct Marks {
  cudaEvent_t* ev = nullptr;
  cudaStream_t stream = nullptr;
  cudaError_t mark(int k) { return ev ? cudaEventRecord(ev[k], stream) : cudaSuccess; }
};

pic_status field_step(Sim* s, int32_t order_p, Marks* mk = nullptr, int base = 0) {
  Marks none;
  Marks& m = mk ? *mk : none;
  pic_status st;
  if (order_p >= 0 && order_p != s->order_tables) {
    if (order_p != 0 && (order_p < 2 || order_p > 512 || (order_p & 1))) {
      set_error("order_p=%d must be 0 (infinite) or even in [2, 512]", order_p);
      return PIC_ERR_ARG;
    }
    if ((st = launch_setup_tables(s, order_p)) != PIC_OK) return st;
  }
  if ((st = fft_forward(s, 4)) != PIC_OK) return st;
  PIC_CUDA(m.mark(base + 1));
  if ((st = dht_forward(s, 4)) != PIC_OK) return st;
  PIC_CUDA(m.mark(base + 2));
  if ((st = launch_psatd(s)) != PIC_OK) return st;
  PIC_CUDA(m.mark(base + 3));
  if ((st = dht_inverse(s)) != PIC_OK) return st;
  PIC_CUDA(m.mark(base + 4));
  if ((st = fft_inverse(s)) != PIC_OK) return st;
  PIC_CUDA(m.mark(base + 5));
  return PIC_OK;
}

// One PIC cycle; with marks, events 0..9 bracket the nine stages of pic_stage.  With the
// moving window on, the push removes the particles that leave through the back edge and,
// when the window moves, the departing column's plasma template is injected after the push
// (inside the gather_push stage) and the column's fields are removed after the field step
// (after the last mark).
pic_status step_once(Sim* s, Marks* mk) {
  Marks none;
  Marks& m = mk ? *mk : none;
  pic_status st;
  WinArgs wa;
  if (s->win.on) {
    wa.on = 1;
    wa.shift = (s->win.cycles + 1) % s->win.period == 0;
    wa.back_col = (int32_t)(s->win.shifts % s->cfg.Nz);
    wa.back_z = wa.back_col * s->cfg.dz;
    wa.flag = reinterpret_cast<int32_t*>(s->win.ws + s->win.flag);
    wa.slot = reinterpret_cast<int32_t*>(s->win.ws + s->win.slot);
    wa.bcnt = reinterpret_cast<int32_t*>(s->win.ws + s->win.bcnt);
  }
  // rho^{n+1} is deposited by the push itself (the sort that follows only reorders
  // particles); with the moving window the mixed forms' injected particles deposit theirs as
  // they are placed, and the FP64 form deposits rho in its own stage after the injection
  const bool fuse_rho = s->cfg.precision != PIC_FP64 || !s->win.on;
  PIC_CUDA(m.mark(0));
  if ((st = launch_gather_push(s, 1, wa, fuse_rho, m.ev ? m.ev[1] : nullptr)) != PIC_OK) return st;
  if (wa.shift && (st = launch_window_inject(s, wa.back_col, fuse_rho)) != PIC_OK) return st;
  PIC_CUDA(m.mark(2));
  if (s->sort_interval <= 1 || s->cycle_idx % s->sort_interval == 0)
    if ((st = launch_sort(s)) != PIC_OK) return st;
  PIC_CUDA(m.mark(3));
  if (!fuse_rho && (st = deposit_rho_with_background(s)) != PIC_OK) return st;
  PIC_CUDA(m.mark(4));
  if ((st = field_step(s, -1, mk, 4)) != PIC_OK) return st;   // marks 5..9
  if (s->win.on) {
    if (wa.shift) {
      if ((st = launch_window_clear(s, wa.back_col)) != PIC_OK) return st;
      s->win.shifts += 1;
    }
    s->win.cycles += 1;
  }
  s->cycle_idx += 1;
  return PIC_OK;
}

#define CHECK_SIM(s)                                              \
  do {                                                            \
    if (!(s)) { set_error("sim handle is NULL"); return PIC_ERR_ARG; } \
  } while (0)

bool valid_tuning(const pic_tuning* t) {
  const bool nt_ok = t->dht_n_tile == 0 || (t->dht_n_tile >= 16 && t->dht_n_tile <= 256 && t->dht_n_tile % 16 == 0);
  const bool ch_ok = t->band_chunk == 512 || t->band_chunk == 1024 || t->band_chunk == 2048;
  return nt_ok && ch_ok;
}

pic_status apply_tuning(Sim* s, int32_t nt, int32_t chunk) {
  s->tune_nt = nt;
  s->tune_chunk = chunk;
  return s->cfg.precision == PIC_FP64 ? PIC_OK : dht_tc_make_maps(s);
}

// Device time of fn() on the handle's stream: one warm-up call, then the best of 3.
template <class F>
pic_status best_of_3(Sim* s, cudaEvent_t e0, cudaEvent_t e1, F&& fn, double* ms) {
  pic_status st = fn();
  if (st != PIC_OK) return st;
  float best = 3.0e38f;
  for (int r = 0; r < 3; ++r) {
    PIC_CUDA(cudaEventRecord(e0, s->stream));
    if ((st = fn()) != PIC_OK) return st;
    PIC_CUDA(cudaEventRecord(e1, s->stream));
    PIC_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    PIC_CUDA(cudaEventElapsedTime(&t, e0, e1));
    best = std::min(best, t);
  }
  *ms = best;
  return PIC_OK;
}

}  // namespace

pic_status step_cycle(Sim* s) { return step_once(s, nullptr); }

}  // namespace pic

using namespace pic;

extern "C" {

const char* pic_last_error(void) { return g_last_error.c_str(); }

pic_status pic_required_bytes(const pic_config* cfg, size_t* bytes) {
  int32_t radix[kMaxRadixPasses], np_;
  pic_status st = validate(cfg, radix, &np_);
  if (st != PIC_OK) return st;
  if (!bytes) { set_error("bytes is NULL"); return PIC_ERR_ARG; }
  *bytes = make_layout(*cfg).total;
  return PIC_OK;
}

pic_status pic_init(const pic_config* cfg, void* workspace, size_t workspace_bytes, void* stream,
                    pic_sim** out) {
  if (!out) { set_error("out is NULL"); return PIC_ERR_ARG; }
  *out = nullptr;
  Sim tmp{};
  pic_status st = validate(cfg, tmp.radix, &tmp.n_radix);
  if (st != PIC_OK) return st;
  Layout L = make_layout(*cfg);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255)) {
    set_error("workspace must be a non-NULL 256-byte aligned device pointer");
    return PIC_ERR_ARG;
  }
  if (workspace_bytes < L.total) {
    set_error("workspace has %zu bytes, %zu required", workspace_bytes, L.total);
    return PIC_ERR_OOM;
  }
  Sim* s = new (std::nothrow) Sim(tmp);
  if (!s) { set_error("host allocation failed"); return PIC_ERR_OOM; }
  s->cfg = *cfg;
  s->lay = L;
  s->stream = reinterpret_cast<cudaStream_t>(stream);
  s->ws = reinterpret_cast<char*>(workspace);
  s->ws_bytes = workspace_bytes;
  s->order_tables = -1;
  s->np = 0;
  s->cur = 0;
  s->cplx_bytes = cfg->precision == PIC_FP64 ? 16 : 8;
  s->tune_nt = 0;
  s->tune_chunk = 1024;
  s->dht_path = PIC_DHT_AUTO;
  s->sort_interval = 1;
  s->cycle_idx = 0;
  s->blue_M = bluestein_length(cfg->Nz, cfg->precision);
  const size_t G = s->grid_elems();
  const size_t cb = s->cplx_bytes;
  auto fail = [&](pic_status e) { delete s; return e; };
  cudaError_t ce;
  if ((ce = cudaMemsetAsync(s->ws + L.E, 0, 6 * G * cb, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if ((ce = cudaMemsetAsync(s->ws + L.Eh, 0, 6 * G * cb, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if (L.ebdw && (ce = cudaMemsetAsync(s->ws + L.ebdw, 0, 6 * G * 16, s->stream)) != cudaSuccess)
    return fail(cuda_status(ce, "memset"));
  if ((ce = cudaMemsetAsync(s->ws + L.rho_prev_h, 0, G * cb, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if ((ce = cudaMemsetAsync(s->ws + L.rho_ion, 0, G * cb, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if ((ce = cudaMemsetAsync(s->ws + L.dep, 0, 4 * G * cb, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if ((ce = cudaMemsetAsync(s->ws + L.err, 0, 256, s->stream)) != cudaSuccess) return fail(cuda_status(ce, "memset"));
  if ((st = fft_configure_device()) != PIC_OK) return fail(st);
  if ((st = dht_tc_configure_device()) != PIC_OK) return fail(st);
  if ((st = dht_tc_make_maps(s)) != PIC_OK) return fail(st);
  if ((st = f64s_configure_device()) != PIC_OK) return fail(st);
  if ((st = f64s_make_maps(s)) != PIC_OK) return fail(st);
  if ((st = particles_configure_device()) != PIC_OK) return fail(st);
  if ((st = launch_setup_twiddles(s)) != PIC_OK) return fail(st);
  if ((st = launch_setup_hankel(s)) != PIC_OK) return fail(st);
  if ((st = launch_setup_tables(s, cfg->order_p)) != PIC_OK) return fail(st);
  if ((st = build_inv_volume(s)) != PIC_OK) return fail(st);
  if ((st = pic_sync(reinterpret_cast<pic_sim*>(s))) != PIC_OK) return fail(st);
  *out = reinterpret_cast<pic_sim*>(s);
  return PIC_OK;
}

pic_status pic_autotune(pic_sim* sim, pic_tuning* out) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  pic_tuning res{s->tune_nt, s->tune_chunk, 0.0, 0.0};
  if (s->cfg.precision != PIC_FP64) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    PIC_CUDA(cudaEventCreate(&e0));
    cudaError_t ce = cudaEventCreate(&e1);
    if (ce != cudaSuccess) { cudaEventDestroy(e0); return cuda_status(ce, "cudaEventCreate"); }
    pic_status st = PIC_OK;
    // DHT: forward (4 source components) + inverse (6 field components) per N tile
    const int nr16 = (s->cfg.Nr + 15) / 16 * 16;
    int last_tiles = -1;
    double best = 3.0e38;
    for (int cand : {256, 128, 64}) {
      const int NT = std::min(cand, nr16);
      const int tiles = (s->cfg.Nr + NT - 1) / NT;
      if (tiles == last_tiles) continue;
      last_tiles = tiles;
      if ((st = apply_tuning(s, cand, s->tune_chunk)) != PIC_OK) break;
      double ms = 0.0;
      st = best_of_3(s, e0, e1, [&]() {
        pic_status q = dht_forward(s, 4);
        return q != PIC_OK ? q : dht_inverse(s);
      }, &ms);
      if (st != PIC_OK) break;
      if (ms < best) { best = ms; res.dht_n_tile = cand; res.dht_ms = ms; }
    }
    // deposit band chunk (the fused J deposit of gather/push uses the same bands)
    if (st == PIC_OK && s->np > 0) {
      best = 3.0e38;
      for (int cand : {512, 1024, 2048}) {
        s->tune_chunk = cand;
        double ms = 0.0;
        st = best_of_3(s, e0, e1, [&]() { return launch_deposit(s, PIC_DEP_J, INT32_MIN, INT32_MAX, nullptr); }, &ms);
        if (st != PIC_OK) break;
        if (ms < best) { best = ms; res.band_chunk = cand; res.deposit_ms = ms; }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != PIC_OK) return st;
    if ((st = apply_tuning(s, res.dht_n_tile, res.band_chunk)) != PIC_OK) return st;
    if ((st = pic_sync(sim)) != PIC_OK) return st;
  }
  if (out) *out = res;
  return PIC_OK;
}

pic_status pic_set_tuning(pic_sim* sim, const pic_tuning* t) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!t || !valid_tuning(t)) {
    set_error("tuning must have dht_n_tile 0 or a multiple of 16 in [16, 256] and band_chunk 512, 1024 or 2048");
    return PIC_ERR_ARG;
  }
  return apply_tuning(s, t->dht_n_tile, t->band_chunk);
}

pic_status pic_set_sort_interval(pic_sim* sim, int32_t interval) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (interval < 1 || interval > 16) {
    set_error("sort interval %d must be in [1, 16]", interval);
    return PIC_ERR_ARG;
  }
  s->sort_interval = interval;
  return PIC_OK;
}

pic_status pic_get_sort_interval(pic_sim* sim, int32_t* interval) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!interval) { set_error("interval is NULL"); return PIC_ERR_ARG; }
  *interval = s->sort_interval;
  return PIC_OK;
}

pic_status pic_set_dht_path(pic_sim* sim, int32_t path) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (path != PIC_DHT_AUTO && path != PIC_DHT_F64_GEMM && path != PIC_DHT_F64_SLICED) {
    set_error("dht path %d is not a pic_dht_path", path);
    return PIC_ERR_ARG;
  }
  if (path == PIC_DHT_F64_SLICED && !f64s_supported(s->cfg)) {
    set_error("the sliced FP64 DHT needs the FP64 form and Nr <= %d", kF64sMaxNr);
    return PIC_ERR_ARG;
  }
  const bool was_dw = eb_dw_active(s);
  s->dht_path = path;
  if (eb_dw_active(s) && !was_dw) return refresh_eb_dw(s);   // E, B came from IEEE rows meanwhile
  return PIC_OK;
}

pic_status pic_get_dht_path(pic_sim* sim, int32_t* path) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!path) { set_error("path is NULL"); return PIC_ERR_ARG; }
  *path = s->dht_path;
  return PIC_OK;
}

pic_status pic_get_tuning(pic_sim* sim, pic_tuning* out) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!out) { set_error("out is NULL"); return PIC_ERR_ARG; }
  *out = pic_tuning{s->tune_nt, s->tune_chunk, 0.0, 0.0};
  return PIC_OK;
}

pic_status pic_fields_to_spectral(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  s->win.pending = 0;   // the spectral state is rebuilt from the (already cleared) real-space fields
  return fields_forward(s);
}

pic_status pic_copy_window(pic_sim* src_sim, int32_t buffer_id, int32_t src_z0, int32_t nz, pic_sim* dst_sim,
                           int32_t dst_z0) {
  Sim* a = reinterpret_cast<Sim*>(src_sim);
  Sim* b = reinterpret_cast<Sim*>(dst_sim);
  CHECK_SIM(a);
  CHECK_SIM(b);
  int ncomp = 0;
  switch (buffer_id) {
    case PIC_BUF_E: case PIC_BUF_B: ncomp = 3; break;
    case PIC_BUF_DEP: ncomp = 4; break;
    case PIC_BUF_RHO_ION: ncomp = 1; break;
    default:
      set_error("buffer %d is not a real-space grid (E, B, DEP or RHO_ION)", buffer_id);
      return PIC_ERR_ARG;
  }
  if (a->cfg.Nr != b->cfg.Nr || a->cfg.Nm != b->cfg.Nm || a->cplx_bytes != b->cplx_bytes) {
    set_error("windows copy between handles of equal Nr, Nm and precision only");
    return PIC_ERR_ARG;
  }
  if (nz < 0 || nz > a->cfg.Nz || nz > b->cfg.Nz) {
    set_error("nz=%d exceeds a grid (source Nz=%d, destination Nz=%d)", nz, a->cfg.Nz, b->cfg.Nz);
    return PIC_ERR_ARG;
  }
  if (nz == 0) return PIC_OK;
  BufView va, vb;
  buffer_view(a, buffer_id, &va);
  buffer_view(b, buffer_id, &vb);
  pic_status st = launch_copy_window(b, a->ws + va.off, a->cfg.Nz, src_z0, b->ws + vb.off, b->cfg.Nz, dst_z0, nz,
                                     ncomp * a->cfg.Nm * a->cfg.Nr);
  if (st == PIC_OK && ncomp == 3 && eb_dw_active(b)) st = refresh_eb_dw(b);
  return st;
}

pic_status pic_destroy(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  if (s && s->diag_host) cudaFreeHost(s->diag_host);
  if (s && s->stage.copy) {   // a staged copy may still be in flight into the caller's buffer
    cudaStreamSynchronize(s->stage.copy);
    cudaEventDestroy(s->stage.copied);
    cudaEventDestroy(s->stage.free_);
    cudaStreamDestroy(s->stage.copy);
  }
  delete s;
  return PIC_OK;
}

pic_status pic_sync(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  int32_t e = 0;
  PIC_CUDA(cudaMemcpyAsync(&e, s->ws + s->lay.err, sizeof(e), cudaMemcpyDeviceToHost, s->stream));
  PIC_CUDA(cudaStreamSynchronize(s->stream));
  if (e & kErrTimeout) { set_error("a device loop hit its iteration cap (error word %d)", e); return PIC_ERR_TIMEOUT; }
  if (e) { set_error("non-finite or out-of-range values on the device (error word %d)", e); return PIC_ERR_NUMERIC; }
  return PIC_OK;
}

pic_status pic_clear_error(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  PIC_CUDA(cudaMemsetAsync(s->ws + s->lay.err, 0, sizeof(int32_t), s->stream));
  return PIC_OK;
}

pic_status pic_selftest_wait_timeout(pic_sim* sim, int32_t max_polls) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (max_polls < 1 || max_polls > (1 << 24)) {
    set_error("max_polls=%d must be in [1, 2^24]", max_polls);
    return PIC_ERR_ARG;
  }
  return launch_wait_selftest(s, (uint32_t)max_polls);
}

pic_status pic_write_particles(pic_sim* sim, const double* const soa[7], const int32_t* id, int64_t n,
                               int32_t on_host) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  if (n < 0 || n > s->cfg.np_capacity) {
    set_error("n=%lld exceeds the capacity %lld", (long long)n, (long long)s->cfg.np_capacity);
    return PIC_ERR_ARG;
  }
  if (n > 0 && (!soa || !id)) { set_error("particle pointers are NULL"); return PIC_ERR_ARG; }
  const cudaMemcpyKind kind = on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  const bool mixed = s->cfg.precision != PIC_FP64;
  const size_t cap = (size_t)s->cfg.np_capacity;
  for (int k = 0; k < 7 && n > 0; ++k) {
    if (!soa[k]) { set_error("particle array %d is NULL", k); return PIC_ERR_ARG; }
    char* dst = mixed ? s->ws + s->lay.stage64 + k * cap * 8 : s->ws + s->lay.part[s->cur][k];
    PIC_CUDA(cudaMemcpyAsync(dst, soa[k], n * 8, kind, s->stream));
  }
  if (n > 0) {
    // ids go straight to their final place (FP64 form) or to the perm scratch (mixed form)
    char* dst = mixed ? s->ws + s->lay.perm_tmp : s->ws + s->lay.pid[s->cur];
    PIC_CUDA(cudaMemcpyAsync(dst, id, n * 4, kind, s->stream));
  }
  s->np = n;
  s->win.on = 0;   // new particles: the window's template and ids no longer apply
  if (mixed) {
    pic_status st = launch_particles_in(s, s->at<int32_t>(s->lay.perm_tmp), n);
    if (st != PIC_OK) return st;
  }
  if (on_host) PIC_CUDA(cudaStreamSynchronize(s->stream));
  return PIC_OK;
}

namespace {
int64_t stage_stride(int64_t n) { return (n + 31) / 32 * 32; }   // doubles per staged array
}   // namespace

pic_status pic_stage_bytes(int64_t n, size_t* bytes) {
  if (!bytes || n < 0) { set_error("pic_stage_bytes: n must be >= 0 and bytes non-NULL"); return PIC_ERR_ARG; }
  const size_t st = (size_t)stage_stride(n);
  *bytes = st * 7 * 8 + st * 4;
  return PIC_OK;
}

pic_status pic_stage_particles(pic_sim* sim, const double* const soa[7], const int32_t* id, int64_t n,
                               void* staging, size_t staging_bytes) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  Sim::StageState& g = s->stage;
  if (g.pending) { set_error("a staged particle set is waiting for pic_take_particles"); return PIC_ERR_STATE; }
  if (n < 0 || n > s->cfg.np_capacity) {
    set_error("n=%lld outside [0, capacity %lld]", (long long)n, (long long)s->cfg.np_capacity);
    return PIC_ERR_ARG;
  }
  size_t need = 0;
  pic_stage_bytes(n, &need);
  if (n > 0) {
    if (!soa || !id) { set_error("particle pointers are NULL"); return PIC_ERR_ARG; }
    for (int k = 0; k < 7; ++k)
      if (!soa[k]) { set_error("particle array %d is NULL", k); return PIC_ERR_ARG; }
    if (!staging || staging_bytes < need || reinterpret_cast<uintptr_t>(staging) % 256 != 0) {
      set_error("staging buffer: %zu bytes at %p, need %zu bytes, 256-byte aligned", staging_bytes, staging, need);
      return PIC_ERR_ARG;
    }
  }
  if (!g.copy) {
    PIC_CUDA(cudaStreamCreateWithFlags(&g.copy, cudaStreamNonBlocking));
    PIC_CUDA(cudaEventCreateWithFlags(&g.copied, cudaEventDisableTiming));
    PIC_CUDA(cudaEventCreateWithFlags(&g.free_, cudaEventDisableTiming));
  }
  const int64_t st = stage_stride(n);
  char* buf = static_cast<char*>(staging);
  // the previous take may still be reading this buffer (an event never recorded is complete)
  PIC_CUDA(cudaStreamWaitEvent(g.copy, g.free_, 0));
  for (int k = 0; k < 7 && n > 0; ++k)
    PIC_CUDA(cudaMemcpyAsync(buf + (size_t)k * st * 8, soa[k], (size_t)n * 8, cudaMemcpyHostToDevice, g.copy));
  if (n > 0) PIC_CUDA(cudaMemcpyAsync(buf + (size_t)7 * st * 8, id, (size_t)n * 4, cudaMemcpyHostToDevice, g.copy));
  PIC_CUDA(cudaEventRecord(g.copied, g.copy));
  g.pending = 1;
  g.n = n;
  g.buf = buf;
  g.stride = st;
  return PIC_OK;
}

pic_status pic_take_particles(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  Sim::StageState& g = s->stage;
  if (!g.pending) { set_error("no staged particle set (pic_stage_particles)"); return PIC_ERR_STATE; }
  g.pending = 0;
  PIC_CUDA(cudaEventSynchronize(g.copied));   // the caller's host arrays are free from here on
  PIC_CUDA(cudaStreamWaitEvent(s->stream, g.copied, 0));
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  const int64_t n = g.n, st = g.stride;
  const double* src = reinterpret_cast<const double*>(g.buf);
  const int32_t* ids = reinterpret_cast<const int32_t*>(g.buf + (size_t)7 * st * 8);
  s->np = n;
  s->win.on = 0;   // new particles: the window's template and ids no longer apply
  if (s->cfg.precision != PIC_FP64) {
    pic_status r = launch_particles_in(s, ids, n, src, st);
    if (r != PIC_OK) return r;
  } else if (n > 0) {
    for (int k = 0; k < 7; ++k)
      PIC_CUDA(cudaMemcpyAsync(s->ws + s->lay.part[s->cur][k], src + (size_t)k * st, (size_t)n * 8,
                               cudaMemcpyDeviceToDevice, s->stream));
    PIC_CUDA(cudaMemcpyAsync(s->ws + s->lay.pid[s->cur], ids, (size_t)n * 4, cudaMemcpyDeviceToDevice, s->stream));
  }
  PIC_CUDA(cudaEventRecord(g.free_, s->stream));
  return PIC_OK;
}

pic_status pic_read_particles(pic_sim* sim, double* const soa[7], int32_t* id, int64_t n,
                              int32_t on_host) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (n < 0 || n > s->np) { set_error("n=%lld exceeds the %lld particles held", (long long)n, (long long)s->np); return PIC_ERR_ARG; }
  const cudaMemcpyKind kind = on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  const bool mixed = s->cfg.precision != PIC_FP64;
  const size_t cap = (size_t)s->cfg.np_capacity;
  if (mixed) {
    pic_status st = launch_particles_out(s, s->at<int32_t>(s->lay.perm_tmp), n);
    if (st != PIC_OK) return st;
  }
  for (int k = 0; k < 7 && n > 0; ++k) {
    const char* src = mixed ? s->ws + s->lay.stage64 + k * cap * 8 : s->ws + s->lay.part[s->cur][k];
    if (soa && soa[k]) PIC_CUDA(cudaMemcpyAsync(soa[k], src, n * 8, kind, s->stream));
  }
  if (id && n > 0) {
    const char* src = mixed ? s->ws + s->lay.perm_tmp : s->ws + s->lay.pid[s->cur];
    PIC_CUDA(cudaMemcpyAsync(id, src, n * 4, kind, s->stream));
  }
  return pic_sync(sim);
}

pic_status pic_num_particles(pic_sim* sim, int64_t* n) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!n) { set_error("n is NULL"); return PIC_ERR_ARG; }
  *n = s->np;
  return PIC_OK;
}

pic_status pic_init_background(pic_sim* sim, int32_t n_neutral) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  const size_t G = s->grid_elems();
  PIC_CUDA(cudaMemsetAsync(s->ws + s->lay.dep, 0, G * s->cplx_bytes, s->stream));
  pic_status st = launch_deposit(s, PIC_DEP_RHO, 0, n_neutral, nullptr);
  if (st != PIC_OK) return st;
  return launch_scale_copy(s, s->ws + s->lay.rho_ion, s->ws + s->lay.dep, -1.0, G);
}

pic_status pic_add_beam_fields(pic_sim* sim, int32_t id_lo, int32_t id_hi, double gamma) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  if (!(gamma >= 1.0)) { set_error("gamma=%g must be >= 1", gamma); return PIC_ERR_ARG; }
  const size_t G = s->grid_elems();
  PIC_CUDA(cudaMemsetAsync(s->ws + s->lay.dep, 0, G * s->cplx_bytes, s->stream));
  pic_status st = launch_deposit(s, PIC_DEP_RHO, id_lo, id_hi, nullptr);
  if (st != PIC_OK) return st;
  if ((st = forward_transform(s, 1)) != PIC_OK) return st;
  return launch_beam_fields(s, s->ws + s->lay.srch, gamma);
}

pic_status pic_init_fields(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  pic_status st = deposit_rho_with_background(s);
  if (st != PIC_OK) return st;
  if ((st = forward_transform(s, 1)) != PIC_OK) return st;
  if ((st = launch_filter_copy(s, s->ws + s->lay.rho_prev_h, s->ws + s->lay.srch)) != PIC_OK) return st;
  if ((st = inverse_transform(s)) != PIC_OK) return st;
  s->fields_ready = 1;
  return PIC_OK;
}

pic_status pic_sort(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  return launch_sort(s);
}

pic_status pic_deposit(pic_sim* sim, int32_t what) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (what & ~(PIC_DEP_RHO | PIC_DEP_J)) { set_error("what=%d has unknown bits", what); return PIC_ERR_ARG; }
  pic_status st;
  if (what & PIC_DEP_RHO) {
    const size_t G = s->grid_elems();
    PIC_CUDA(cudaMemcpyAsync(s->ws + s->lay.dep, s->ws + s->lay.rho_ion, G * s->cplx_bytes,
                             cudaMemcpyDeviceToDevice, s->stream));
  }
  if ((st = launch_deposit(s, what, INT32_MIN, INT32_MAX, nullptr)) != PIC_OK) return st;
  return PIC_OK;
}

pic_status pic_gather_push(pic_sim* sim, int32_t fuse_current) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  return launch_gather_push(s, fuse_current);
}

pic_status pic_field_step(pic_sim* sim, int32_t order_p) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  return field_step(s, order_p);
}

pic_status pic_forward_transform(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  return forward_transform(s, 4);
}

pic_status pic_psatd(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  return launch_psatd(s);
}

pic_status pic_inverse_transform(pic_sim* sim) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  return inverse_transform(s);
}

pic_status pic_step(pic_sim* sim, int32_t n_steps) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (n_steps < 0) { set_error("n_steps=%d < 0", n_steps); return PIC_ERR_ARG; }
  if (!s->fields_ready) { set_error("pic_init_fields must run before stepping"); return PIC_ERR_STATE; }
  for (int32_t k = 0; k < n_steps; ++k) {
    pic_status st = step_once(s, nullptr);
    if (st != PIC_OK) return st;
  }
  return PIC_OK;
}

pic_status pic_step_timed(pic_sim* sim, int32_t n_steps, double* stage_ms) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (n_steps < 1 || n_steps > 4096 || !stage_ms) { set_error("n_steps must be in [1, 4096] and stage_ms non-NULL"); return PIC_ERR_ARG; }
  if (!s->fields_ready) { set_error("pic_init_fields must run before stepping"); return PIC_ERR_STATE; }
  const int per = PIC_NSTAGES + 1;
  const size_t nev = (size_t)n_steps * per;
  cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[nev];
  if (!ev) { set_error("host allocation failed"); return PIC_ERR_OOM; }
  size_t made = 0;
  pic_status st = PIC_OK;
  for (; made < nev; ++made) {
    cudaError_t e = cudaEventCreate(&ev[made]);
    if (e != cudaSuccess) { st = cuda_status(e, "cudaEventCreate"); break; }
  }
  for (int32_t k = 0; st == PIC_OK && k < n_steps; ++k) {
    Marks mk;
    mk.ev = ev + (size_t)k * per;
    mk.stream = s->stream;
    st = step_once(s, &mk);
  }
  if (st == PIC_OK) {
    cudaError_t e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) st = cuda_status(e, "cudaStreamSynchronize");
  }
  if (st == PIC_OK) {
    for (int i = 0; i <= PIC_NSTAGES; ++i) stage_ms[i] = 0.0;
    for (int32_t k = 0; k < n_steps && st == PIC_OK; ++k) {
      for (int i = 0; i < PIC_NSTAGES; ++i) {
        float ms = 0.f;
        cudaError_t e = cudaEventElapsedTime(&ms, ev[(size_t)k * per + i], ev[(size_t)k * per + i + 1]);
        if (e != cudaSuccess) { st = cuda_status(e, "cudaEventElapsedTime"); break; }
        stage_ms[i] += ms;
      }
    }
    float tot = 0.f;
    if (st == PIC_OK) {
      cudaError_t e = cudaEventElapsedTime(&tot, ev[0], ev[nev - 1]);
      if (e != cudaSuccess) st = cuda_status(e, "cudaEventElapsedTime");
      stage_ms[PIC_NSTAGES] = tot;
    }
  }
  for (size_t i = 0; i < made; ++i) cudaEventDestroy(ev[i]);
  delete[] ev;
  if (st != PIC_OK) return st;
  return pic_sync(sim);
}

pic_status pic_diagnostics(pic_sim* sim, int32_t id_lo, int32_t id_hi, pic_diag* out,
                           double* slice_sigma, int32_t max_slices) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!out) { set_error("out is NULL"); return PIC_ERR_ARG; }
  pic_status st = launch_diag(s, id_lo, id_hi, out, slice_sigma, max_slices);
  if (st != PIC_OK) return st;
  return pic_sync(sim);
}

pic_status pic_buffer_bytes(pic_sim* sim, int32_t buffer_id, size_t* bytes) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  BufView v;
  if (!bytes || !buffer_view(s, buffer_id, &v)) { set_error("unknown buffer %d", buffer_id); return PIC_ERR_ARG; }
  *bytes = v.bytes;
  return PIC_OK;
}

pic_status pic_copy_buffer(pic_sim* sim, int32_t buffer_id, void* dst, size_t bytes, int32_t dst_on_host) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  BufView v;
  if (!buffer_view(s, buffer_id, &v)) { set_error("unknown buffer %d", buffer_id); return PIC_ERR_ARG; }
  if (!dst || bytes != v.bytes) { set_error("buffer %d has %zu bytes, %zu given", buffer_id, v.bytes, bytes); return PIC_ERR_ARG; }
  PIC_CUDA(cudaMemcpyAsync(dst, s->ws + v.off, bytes,
                           dst_on_host ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, s->stream));
  if (dst_on_host) return pic_sync(sim);
  return PIC_OK;
}

pic_status pic_load_buffer(pic_sim* sim, int32_t buffer_id, const void* src, size_t bytes, int32_t src_on_host) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (pic_status fs = launch_window_flush(s)) return fs;   // pending window-column subtraction
  BufView v;
  if (!buffer_view(s, buffer_id, &v)) { set_error("unknown buffer %d", buffer_id); return PIC_ERR_ARG; }
  if (buffer_id == PIC_BUF_KEYS || buffer_id == PIC_BUF_PERM) { set_error("buffer %d is read-only", buffer_id); return PIC_ERR_ARG; }
  if (!src || bytes != v.bytes) { set_error("buffer %d has %zu bytes, %zu given", buffer_id, v.bytes, bytes); return PIC_ERR_ARG; }
  PIC_CUDA(cudaMemcpyAsync(s->ws + v.off, src, bytes,
                           src_on_host ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s->stream));
  if (src_on_host) PIC_CUDA(cudaStreamSynchronize(s->stream));
  if (buffer_id == PIC_BUF_E || buffer_id == PIC_BUF_B) {
    s->fields_ready = 1;
    if (eb_dw_active(s)) return refresh_eb_dw(s);
  }
  return PIC_OK;
}

pic_status pic_window_required_bytes(pic_sim* sim, int64_t n_plasma, size_t* bytes) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!bytes || n_plasma < 0 || n_plasma > s->cfg.np_capacity) {
    set_error("bytes is NULL or n_plasma=%lld outside [0, capacity]", (long long)n_plasma);
    return PIC_ERR_ARG;
  }
  *bytes = window_layout(s, n_plasma, nullptr);
  return PIC_OK;
}

pic_status pic_window_setup(pic_sim* sim, int64_t n_plasma, int32_t period, int64_t n_reserve, void* workspace,
                            size_t workspace_bytes) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (s->win.on) { set_error("the moving window is already on"); return PIC_ERR_ARG; }
  if (period < 1) { set_error("period=%d must be >= 1", period); return PIC_ERR_ARG; }
  if (n_plasma < 0 || n_plasma > s->np) {
    set_error("n_plasma=%lld outside [0, %lld particles held]", (long long)n_plasma, (long long)s->np);
    return PIC_ERR_ARG;
  }
  if (n_reserve < 0 || s->np + n_reserve > s->cfg.np_capacity) {
    set_error("n_reserve=%lld: %lld + reserve exceeds the capacity %lld", (long long)n_reserve, (long long)s->np,
              (long long)s->cfg.np_capacity);
    return PIC_ERR_ARG;
  }
  WindowState w;
  const size_t need = window_layout(s, n_plasma, &w);
  if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 255) || workspace_bytes < need) {
    set_error("window workspace must be 256-byte aligned with >= %zu bytes", need);
    return PIC_ERR_ARG;
  }
  // the ids held must be exactly 0 .. np-1 (slots are found by id)
  const int64_t np = s->np;
  std::vector<int32_t> ids, cols;
  std::vector<char> seen;
  try {
    ids.resize((size_t)np);
    seen.assign((size_t)np, 0);
    cols.resize((size_t)n_plasma);
  } catch (...) {
    set_error("host allocation failed");
    return PIC_ERR_OOM;
  }
  const bool mixed = s->cfg.precision != PIC_FP64;
  const char* id_src = mixed ? s->ws + s->lay.pf[s->cur][kPfId] : s->ws + s->lay.pid[s->cur];
  if (np > 0) {
    PIC_CUDA(cudaMemcpyAsync(ids.data(), id_src, np * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream));
    PIC_CUDA(cudaStreamSynchronize(s->stream));
  }
  for (int64_t i = 0; i < np; ++i) {
    const int32_t k = ids[i];
    if (k < 0 || k >= np || seen[k]) {
      set_error("window: particle ids must be exactly 0 .. np-1 (id %d at %lld)", k, (long long)i);
      return PIC_ERR_ARG;
    }
    seen[k] = 1;
  }
  w.ws = reinterpret_cast<char*>(workspace);
  w.period = period;
  w.n_tpl = n_plasma;
  s->win = w;
  pic_status st = window_take_template(s, cols.data());
  if (st != PIC_OK) return st;
  // template ids grouped by column, increasing id within a column (counting sort)
  const int Nz = s->cfg.Nz;
  std::vector<int32_t> start((size_t)Nz + 1, 0), order;
  try {
    order.resize((size_t)std::max<int64_t>(n_plasma, 1));
  } catch (...) {
    set_error("host allocation failed");
    return PIC_ERR_OOM;
  }
  for (int64_t k = 0; k < n_plasma; ++k) start[cols[k] + 1] += 1;
  for (int c = 0; c < Nz; ++c) start[c + 1] += start[c];
  std::vector<int32_t> cursor(start.begin(), start.end() - 1);
  for (int64_t k = 0; k < n_plasma; ++k) order[cursor[cols[k]]++] = (int32_t)k;
  if (n_plasma > 0)
    PIC_CUDA(cudaMemcpy(s->win.ws + s->win.colids, order.data(), n_plasma * sizeof(int32_t), cudaMemcpyHostToDevice));
  PIC_CUDA(cudaMemsetAsync(s->win.ws + s->win.dropped, 0, 8, s->stream));
  if ((st = launch_window_reserve(s, n_reserve)) != PIC_OK) return st;
  // records of the inactive particles (the reserve and any particle held with w = 0)
  PIC_CUDA(cudaMemsetAsync(s->win.ws + s->win.flag, 0, (size_t)s->np * sizeof(int32_t), s->stream));
  PIC_CUDA(cudaMemsetAsync(s->win.ws + s->win.bcnt, 0, ((size_t)s->np / 1024 + 2) * sizeof(int32_t), s->stream));
  if ((st = launch_window_mark_all(s)) != PIC_OK) return st;
  s->win.col_start_host = std::move(start);
  s->win.n_ids = s->np;
  s->win.cycles = 0;
  s->win.shifts = 0;
  s->win.on = 1;
  return pic_sync(sim);
}

pic_status pic_window_state(pic_sim* sim, pic_window_info* out) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!s->win.on) { set_error("the moving window is not set up"); return PIC_ERR_STATE; }
  if (!out) { set_error("out is NULL"); return PIC_ERR_ARG; }
  unsigned long long dropped = 0;
  PIC_CUDA(cudaMemcpyAsync(&dropped, s->win.ws + s->win.dropped, 8, cudaMemcpyDeviceToHost, s->stream));
  PIC_CUDA(cudaStreamSynchronize(s->stream));
  out->cycles = s->win.cycles;
  out->shifts = s->win.shifts;
  out->back_column = (int32_t)(s->win.shifts % s->cfg.Nz);
  out->period = s->win.period;
  out->dropped = (int64_t)dropped;
  out->n_template = s->win.n_tpl;
  return PIC_OK;
}

pic_status pic_launch_count(pic_sim* sim, int64_t* launches) {
  Sim* s = reinterpret_cast<Sim*>(sim);
  CHECK_SIM(s);
  if (!launches) { set_error("launches is NULL"); return PIC_ERR_ARG; }
  *launches = s->launches;
  return PIC_OK;
}

}  // extern "C"
