// A0: channel frequencies and the integer delay table of Eq. 1.
//
// The table is computed on the GPU in binary64 with explicitly rounded
// intrinsics (no fused multiply-add), in the fixed operation order
//   f_c     = f_lo + (c + 1/2) * (bw / nchan)
//   inv_c   = 1 / (f_c * f_c),  inv_ref = 1 / (f_ref * f_ref)
//   v       = ((4148.808 * DM) * (inv_c - inv_ref)) / t_samp
//   delay   = floor(v + 1/2)
// so that the integer shifts are reproducible bit for bit.  f_ref is the
// highest channel centre; channel centres are monotone in c, so it is the
// centre of channel 0 or of channel nchan - 1.
#include "tp_common.cuh"

namespace tp {

namespace {

constexpr double kDispersionConstant = 4148.808;  // s MHz^2 (Eq. 1)

__device__ __forceinline__ double centre(double f_lo, double df, int c) {
  return __dadd_rn(f_lo, __dmul_rn((double)c + 0.5, df));
}

__global__ void delay_table_kernel(int nchan, double f_lo, double bw, double t_samp,
                                   const double* __restrict__ dm, int ndm,
                                   int32_t* __restrict__ delay, int* __restrict__ err) {
  const double df = __ddiv_rn(bw, (double)nchan);
  const double f0 = centre(f_lo, df, 0);
  const double f1 = centre(f_lo, df, nchan - 1);
  const double f_ref = f0 > f1 ? f0 : f1;
  const double inv_ref = __ddiv_rn(1.0, __dmul_rn(f_ref, f_ref));
  const int64_t n = (int64_t)nchan * ndm;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int d = (int)(i / nchan);
    const int c = (int)(i - (int64_t)d * nchan);
    const double f = centre(f_lo, df, c);
    const double inv_c = __ddiv_rn(1.0, __dmul_rn(f, f));
    const double v = __ddiv_rn(__dmul_rn(__dmul_rn(kDispersionConstant, dm[d]),
                                         __dsub_rn(inv_c, inv_ref)),
                               t_samp);
    const double r = floor(__dadd_rn(v, 0.5));
    if (!(r >= 0.0) || r > 2147483647.0) {
      atomicExch(err, 1);
      delay[i] = 0;
    } else {
      delay[i] = (int32_t)r;
    }
  }
}

}  // namespace

cudaError_t launch_delay_table(int nchan, double f_lo, double bw, double t_samp, const double* dm,
                               int ndm, int32_t* delay, int* err_flag, cudaStream_t s) {
  const int64_t n = (int64_t)nchan * ndm;
  int blocks = (int)((n + 255) / 256);
  if (blocks > 152 * 8) blocks = 152 * 8;
  if (blocks < 1) blocks = 1;
  delay_table_kernel<<<blocks, 256, 0, s>>>(nchan, f_lo, bw, t_samp, dm, ndm, delay, err_flag);
  return cudaGetLastError();
}

}  // namespace tp
