// Internal declarations shared by the translation units of libpsatd_rz.so.
//
// Paper: Jalas et al., arXiv:1611.05712 -- quasi-cylindrical arbitrary-order PSATD
// PIC cycle (section "Finite order pseudo-spectral solvers").  The public contract is
// include/psatd_rz.h; this header holds the device-side layout and the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/psatd_rz.h"

namespace pic {

// SI constants, CODATA 2018; mu0 is tied to eps0 and c so that mu0 eps0 c^2 = 1.
constexpr double kC = 299792458.0;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * kC * kC);
constexpr double kPi = 3.14159265358979323846;
constexpr double kPinvRcond = 1e-3;   // singular values <= rcond * sigma_max are dropped
constexpr double kSmallX = 0.25;      // omega*dt below which the PSATD coefficients use series
constexpr double kSliceLen = 0.5e-6;  // slice length of the slice energy spread [m]

constexpr int kMaxModes = 4;
constexpr int kMaxNr = 1024;
constexpr int kMaxRadixPasses = 16;

// Device error word bits.
enum : int32_t { kErrNumeric = 1, kErrTimeout = 2, kErrRange = 4 };

// Device workspace layout, all offsets in bytes from the workspace base.
struct Layout {
  size_t E, B, Eh, Bh, dep, srch, tmp, rho_prev_h, rho_ion;   // grids
  size_t kperp, binv, mfwd, svd_w, svd_v, svd_d;                // DHT tables and scratch
  size_t kzmod, tz, tr, coef;                                    // PSATD tables
  size_t twp;        // per-pass twiddle tables of the row FFT (radix-8 or mixed-radix plan)
  size_t twp_dw;     // the same as double words (hi, lo float pairs), FP64 form
  // FP64 form with power-of-two Nz (0 otherwise): E, B as double words, [6][Nm][Nr][Nz]
  // float4 (re.hi, re.lo, im.hi, im.lo), written beside E, B by the inverse row FFT and read
  // by the gather
  size_t ebdw;
  size_t part[2][7], pid[2];                                     // particles (double buffer)
  size_t keys, perm, perm_tmp, count, start, scan_blk, big_list, big_count;
  size_t diag_acc, err;
  // mixed-precision form only (0 otherwise): float copies of the tables, the split DHT
  // matrices, FP32 cell-relative particles and an FP64 staging area for particle IO
  size_t coef_f, kperp_f, kzmod_f, tz_f, tr_f, twp_f;
  size_t mfwd_hi, mfwd_lo, binv_hi, binv_lo;   // TF32 form: hi/lo planes; BF16 form: *_hi = 3 planes
  size_t pf[2][13];  // iz, fz, ixy (packed int16 x, y cells), fx, fy, u/c hi (3), u/c lo (3), w, id
  size_t stage64;    // 7 x capacity float64
  size_t ebt;        // E, B with r fastest: [6][Nm][Nz][Nr] complex float (gather layout)
  // Nz that is not 7-smooth (Bluestein, 0 otherwise): twiddles of the power-of-two length M,
  // the chirp w_n (Nz), the chirp filter's spectrum (M), float copies
  size_t twm, twm_f, chirp, chirp_f, bspec, bspec_f;
  // FP64 form with Nr <= 256: the sliced tensor-core DHT (BF16 slice planes of the matrices
  // and of the current panels, their row and column exponents)
  size_t f64s_mat, f64s_rowexp, f64s_panel, f64s_colexp;
  size_t total;
};

// Power-of-two convolution length M >= 2 Nz - 1 of Bluestein's algorithm for an Nz that is
// not 7-smooth; 0 when Nz is 7-smooth (direct FFT) or when M exceeds the row FFT's limit
// (4096 FP64, 8192 float).
int bluestein_length(int Nz, int precision);

// Row pitch (floats) of the split DHT matrices of the mixed form: Nr rounded up to a
// multiple of 4 so that rows start on 16-byte boundaries (tensor-memory-access copies).
inline int split_pitch(int Nr) { return (Nr + 3) / 4 * 4; }
// Row pitch (elements) of the BF16 planes of the BF16 form: Nr rounded up to a multiple of 8.
inline int split_pitch_b16(int Nr) { return (Nr + 7) / 8 * 8; }

// FP32 particle array indices of the mixed form: z = (iz + fz) dz, x = (ix + fx) dr,
// y = (iy + fy) dr with fz, fx, fy in [0, 1) and (ix, iy) two int16 packed in one int32;
// u/c = hi + lo per component (float pairs, |lo| <= ulp(hi)/2).
enum {
  kPfIz = 0, kPfFz, kPfIxy, kPfFx, kPfFy, kPfUx, kPfUy, kPfUz, kPfUxLo, kPfUyLo, kPfUzLo, kPfW, kPfId,
  kPfCount
};

// Push arguments of the moving window (pic_window_setup): with on = 1 the push removes
// the particles that end behind the back edge; shift = 1 when the window moves at the end
// of this cycle.
struct WinArgs {
  int32_t on = 0, shift = 0, back_col = 0;
  double back_z = 0.0;   // back_col * dz
  // a particle the push removes is recorded for the injections:
  // flag[id] = 1, slot[id] = array index, bcnt[id / 1024] += 1
  int32_t* flag = nullptr;
  int32_t* slot = nullptr;
  int32_t* bcnt = nullptr;
};

// Moving-window state of a handle; offsets are bytes into the caller's window workspace.
struct WindowState {
  int32_t on = 0, period = 1;
  int32_t pending = 0;     // the last departed column's spectral subtraction is not applied yet
  int64_t cycles = 0, shifts = 0;
  int64_t n_tpl = 0;       // template particles (ids < n_tpl)
  int64_t n_ids = 0;       // ids 0 .. n_ids-1 held (particles plus reserve)
  char* ws = nullptr;
  size_t tpl, colids, flag, slot, bcnt, bstart, dropped, colv, hv, ph, hvf, phf;   // hvf, phf: float copies
  std::vector<int32_t> col_start_host;   // [Nz + 1] template offsets per column
};

struct Sim {
  pic_config cfg;
  Layout lay;
  cudaStream_t stream;
  char* ws;
  size_t ws_bytes;
  int32_t order_tables;    // order p the coefficient tables were built for
  int64_t np;              // particles held
  int cur;                 // which particle buffer is current
  int fields_ready;
  int64_t launches;        // kernels launched by this handle (host-side count)
  int32_t n_radix;
  int32_t radix[kMaxRadixPasses];
  int32_t blue_M;          // Bluestein convolution length (0: direct FFT of length Nz)
  size_t cplx_bytes;       // 16 (FP64) or 8 (mixed)
  int32_t tune_nt;         // mixed-form DHT N tile (0: built-in rule), see pic_set_tuning
  int32_t tune_chunk;      // particles per CTA of the band kernels
  int32_t dht_path;        // FP64 form: pic_dht_path (automatic, SIMT GEMM or sliced tensor cores)
  int32_t sort_interval;   // pic_step sorts on every sort_interval-th cycle (1: every cycle)
  int64_t cycle_idx;       // cycles pic_step has run on this handle
  // mixed forms: encoded 2-D tensor maps (CUtensorMap, 128 B each) of the split DHT
  // matrices, [matrix id][plane] (TF32: hi, lo; BF16: three pieces), built at init
  struct alignas(64) TensorMapBytes {
    unsigned char b[128];
  } tmaps[2 * kMaxModes * 3][3];
  TensorMapBytes f64s_maps[2];   // FP64 form: panel planes, matrix planes (sliced DHT)
  WindowState win;
  double* diag_host = nullptr;   // pinned host copy of the diagnostics results (first use)
  // staged particle input (pic_stage_particles / pic_take_particles): a copy stream and
  // two events, created on first use
  struct StageState {
    cudaStream_t copy = nullptr;
    cudaEvent_t copied = nullptr;   // the staged copy has landed
    cudaEvent_t free_ = nullptr;    // the last take has read its staging buffer
    int pending = 0;
    int64_t n = 0;
    char* buf = nullptr;            // caller's device staging buffer
    int64_t stride = 0;             // doubles per array in buf
  } stage;

  template <typename T> T* at(size_t off) const { return reinterpret_cast<T*>(ws + off); }
  size_t grid_elems() const { return (size_t)cfg.Nm * cfg.Nr * cfg.Nz; }
};

// Error reporting (thread-local text, see pic_last_error).
void set_error(const char* fmt, ...);
pic_status cuda_status(cudaError_t e, const char* what);

#define PIC_CUDA(call)                                                     \
  do {                                                                     \
    cudaError_t e__ = (call);                                              \
    if (e__ != cudaSuccess) return ::pic::cuda_status(e__, #call);         \
  } while (0)

#define PIC_LAUNCHED(sim)                                                  \
  do {                                                                     \
    (sim)->launches++;                                                     \
    cudaError_t e__ = cudaGetLastError();                                  \
    if (e__ != cudaSuccess) return ::pic::cuda_status(e__, "kernel launch"); \
  } while (0)

// ---- launchers (setup.cu) ----
pic_status launch_setup_hankel(Sim* s);          // zeros, B_p, pinv(B_p)
pic_status launch_setup_tables(Sim* s, int32_t order_p);   // [k_z]_p and PSATD coefficients
pic_status launch_setup_twiddles(Sim* s);
pic_status convert_hankel_tables(Sim* s);                    // mixed form: float/split copies
pic_status convert_psatd_tables(Sim* s);

// ---- launchers (fft.cu) ----
// Row transform descriptor: out[c] = FFT(ca*in[srcA] + cb*in[srcB]) (inverse: iFFT).
struct RowCombine {
  int32_t n_out;
  int32_t srcA[6], srcB[6];   // srcB < 0: none
  double caRe[6], caIm[6], cbRe[6], cbIm[6];
  // filled by launch_fft_rows from the coefficients above: kind 0 real, 1 imaginary, 2
  // general; unit +1 / -1 when the coefficient is +-1 (kind 0) or +-i (kind 1), else 0;
  // float copies for the float rows (no float64 conversions in those kernels)
  int8_t kindA[6], kindB[6], unitA[6], unitB[6];
  float fcaRe[6], fcaIm[6], fcbRe[6], fcbIm[6];
  // optional second destination of the double-word rows (power-of-two FP64 rows): the
  // outputs as float4 (re.hi, re.lo, im.hi, im.lo) in the layout of `out`; null for none
  void* out_dw;
};
pic_status launch_fft_rows(Sim* s, const void* in, void* out, const RowCombine& rc, bool inverse);
// The double-word copy of E, B is kept (FP64 form, power-of-two rows in double words).
bool eb_dw_active(const Sim* s);
pic_status refresh_eb_dw(Sim* s);       // rebuild it from E, B after a write of those
pic_status fft_configure_device();      // once per device, before any FFT launch
bool fft_is_pow2(int N);                // rows of power-of-two length use the radix-8 kernel

// ---- launchers (dht.cu) ----
// out[b] = A[b] (Nr x Nr, row-major [out][red]) * in[b] (Nr x 2Nz reals).  FP64 form: A[b]
// points at the float64 matrix.  Mixed forms: mat[b] names the split matrix whose tensor
// maps the tcgen05 kernel reads (fwd: m*3+slot, inv: kMaxModes*3 + m*3+slot); X, Y float.
struct DhtBatch {
  int32_t n;
  const void* A[24];
  const void* X[24];
  void* Y[24];
  int16_t mat[24];
};
// The DHT of the current precision form (FP64 SIMT, or 3-term TF32 on tcgen05).
pic_status launch_dht(Sim* s, const DhtBatch& b);
// FP64 Y = A X with A Nr x Nr and X Nr x ncols (setup products and the FP64 DHT).
pic_status launch_gemm_f64(Sim* s, const DhtBatch& b, int ncols);
// Mixed forms: Y = A X with split products on tcgen05 (dht_tc.cu); A from the tensor maps.
pic_status launch_dht_tc(Sim* s, const DhtBatch& b);
pic_status dht_tc_configure_device();   // once per device, before any tcgen05 DHT launch
pic_status dht_tc_make_maps(Sim* s);     // once per handle: tensor maps of the split matrices
pic_status launch_wait_selftest(Sim* s, uint32_t max_polls);   // bounded wait that times out
void* tensor_map_encoder();              // the driver's cuTensorMapEncodeTiled, or null
int dht_tc_sm_count();                   // SMs of the current device
// FP64 form, Nr <= kF64sMaxNr: the DHT from exact BF16 slice products on tcgen05 (dht_f64s.cu)
constexpr int kF64sSlices = 7;
constexpr int kF64sMaxNr = 256;
bool f64s_supported(const pic_config& c);
bool f64s_active(const Sim* s);
pic_status f64s_configure_device();
pic_status f64s_make_maps(Sim* s);
pic_status launch_f64s_setup(Sim* s);
pic_status launch_dht_f64s(Sim* s, const DhtBatch& b);

// ---- launchers (psatd.cu) ----
// PSATD update; with a pending window-column removal it is applied to Eh, Bh on load.
pic_status launch_psatd(Sim* s);
pic_status launch_beam_fields(Sim* s, const void* rho_h, double gamma);  // adds to Eh, Bh
pic_status launch_filter_copy(Sim* s, void* dst, const void* src);        // dst = T * src
pic_status launch_scale_copy(Sim* s, void* dst, const void* src, double a, size_t n_cplx);

// ---- launchers (domain.cu) ----
// dst rows [row][dst_z0 + t mod dst_nz] = src rows [row][src_z0 + t mod src_nz], t < nz, for
// `rows` complex rows of either element size (cplx_bytes of dst), on dst's stream.
pic_status launch_copy_window(Sim* dst_sim, const char* src, int src_nz, int src_z0, char* dst, int dst_nz,
                              int dst_z0, int nz, int rows);

// ---- launchers (particles.cu) ----
pic_status launch_sort(Sim* s);
pic_status launch_deposit(Sim* s, int32_t what, int32_t id_lo, int32_t id_hi, void* rho_out);
// fuse_rho (mixed forms): also deposit rho^{n+1} + background at x^{n+1}.
// after_layout (optional): recorded on the handle's stream once the gather layout is built
// (before the particle kernel), for the stage timing.
pic_status launch_gather_push(Sim* s, int32_t fuse_current, const WinArgs& wa = WinArgs{}, bool fuse_rho = false,
                              cudaEvent_t after_layout = nullptr);
pic_status launch_diag(Sim* s, int32_t id_lo, int32_t id_hi, pic_diag* out, double* slice_sigma,
                       int32_t max_slices);
pic_status build_inv_volume(Sim* s);                        // once, at init
pic_status particles_configure_device();                    // once per device
// mixed: float64 SoA (7 arrays of `stride` doubles from src; stage64 with the capacity as
// stride when src is null) -> FP32
pic_status launch_particles_in(Sim* s, const int32_t* id_dev, int64_t n, const double* src = nullptr,
                               int64_t stride = 0);
pic_status launch_particles_out(Sim* s, int32_t* id_dev, int64_t n);        // mixed: FP32 -> stage64

// ---- moving window (particles.cu: particle side; window.cu: field side) ----
// Byte offsets of the window workspace for a template of n_tpl particles.
size_t window_layout(const Sim* s, int64_t n_tpl, WindowState* w);
// Append n_reserve inactive particles (ids np ..); np grows by n_reserve.
pic_status launch_window_reserve(Sim* s, int64_t n_reserve);
// Template of the particles with id < n_tpl (by id) into the window workspace; keys_host
// receives the column of each template particle.  Synchronises.
pic_status window_take_template(Sim* s, int32_t* keys_host);
// Record every inactive particle for the injections (flag, slot, per-block count).
pic_status launch_window_mark_all(Sim* s);
// Template of column `column` into the inactive particles, smallest id first; with
// deposit_rho (mixed forms, whose push deposited rho^{n+1}) the placed particles' rho too.
pic_status launch_window_inject(Sim* s, int column, bool deposit_rho);
// Departing column removed from E, B: real space zeroed now; the subtraction of its transform
// from Eh, Bh is left pending (applied by the next PSATD or by launch_window_flush).
pic_status launch_window_clear(Sim* s, int column);
// Apply a pending spectral subtraction now (before Eh, Bh are read or changed elsewhere).
pic_status launch_window_flush(Sim* s);

}  // namespace pic
