// Window copies between simulation handles along z, for domain decomposition with guard
// cells (sections "Finite order pseudo-spectral solvers" and "Conclusion": a stencil of
// finite order p reaches only a finite number of cells, so a subdomain extended by that
// many guard cells can be advanced with its own Fourier transform).
#include "pic_internal.cuh"

namespace pic {
namespace {

// One thread per (row, t): dst[row][(dst_z0 + t) mod dst_nz] = src[row][(src_z0 + t) mod src_nz].
template <typename C2>
__global__ void k_copy_window(const C2* __restrict__ src, int src_nz, int src_z0, C2* __restrict__ dst, int dst_nz,
                              int dst_z0, int nz, int rows) {
  const int row = blockIdx.y;
  if (row >= rows) return;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nz; t += gridDim.x * blockDim.x) {
    int zs = (src_z0 + t) % src_nz;
    if (zs < 0) zs += src_nz;
    int zd = (dst_z0 + t) % dst_nz;
    if (zd < 0) zd += dst_nz;
    dst[(size_t)row * dst_nz + zd] = src[(size_t)row * src_nz + zs];
  }
}

}  // namespace

pic_status launch_copy_window(Sim* s, const char* src, int src_nz, int src_z0, char* dst, int dst_nz, int dst_z0,
                              int nz, int rows) {
  if (rows <= 0 || nz <= 0) return PIC_OK;
  const int threads = 256;
  dim3 grid((nz + threads - 1) / threads, rows);
  if (s->cplx_bytes == 16)
    k_copy_window<double2><<<grid, threads, 0, s->stream>>>(reinterpret_cast<const double2*>(src), src_nz, src_z0,
                                                            reinterpret_cast<double2*>(dst), dst_nz, dst_z0, nz, rows);
  else
    k_copy_window<float2><<<grid, threads, 0, s->stream>>>(reinterpret_cast<const float2*>(src), src_nz, src_z0,
                                                           reinterpret_cast<float2*>(dst), dst_nz, dst_z0, nz, rows);
  PIC_LAUNCHED(s);
  return PIC_OK;
}

}  // namespace pic
