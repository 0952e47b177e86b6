// A1-A3: bandpass statistics, channel thresholding and spectrum thresholding
// ("Bandpass Correction", "Channel Thresholding" and "Spectrum Thresholding"
// of Sec. 2.2.1).
//
// Kernel chunk_stats (one CTA per channel): every W_c-sample chunk of the
// window is summed by one warp.  Float data are summed as (x - p) with a
// per-channel pivot p near the mean (the FP32 mean of the first 64 samples),
// in FP32 inside sub-chunks of at most 256 samples and in FP64 above that;
// 8-bit data are summed exactly in integers.  The per-chunk sums go to global
// scratch; the channel totals give mu_c and sigma_c, and each chunk is then
// tested against tau_c sigma_c sqrt(n_k).
// Kernel dilate: flag = own exceedance | time neighbours (| channel
// neighbours); per-channel flagged-chunk counts.  Kernel spectrum_threshold
// (one CTA per 256 samples): the sum over channels of the corrected samples of
// unflagged chunks, compared with tau_s sqrt(sum_c sigma_c^2).
#include <cstdint>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

template <int DT>
__device__ __forceinline__ float load_as_float(const void* x, int64_t i);
template <>
__device__ __forceinline__ float load_as_float<TP_F32>(const void* x, int64_t i) {
  return __ldg(static_cast<const float*>(x) + i);
}
template <>
__device__ __forceinline__ float load_as_float<TP_F16>(const void* x, int64_t i) {
  unsigned short h = __ldg(static_cast<const unsigned short*>(x) + i);
  float f;
  asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
  return f;
}
template <>
__device__ __forceinline__ float load_as_float<TP_BF16>(const void* x, int64_t i) {
  unsigned short h = __ldg(static_cast<const unsigned short*>(x) + i);
  return __uint_as_float((unsigned)h << 16);
}

__device__ __forceinline__ unsigned load_u8(const void* x, int64_t i) {
  return __ldg(static_cast<const unsigned char*>(x) + i);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Chunk sums (float data).  Writes chunk_sums[c][k] = {sum(x - p), sum((x - p)^2)}
// and the channel statistics.
template <int DT>
__global__ void __launch_bounds__(kThreads) chunk_stats_float(RfiArgs a, double2* chunk_sums) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)c * a.pitch;
  __shared__ float s_pivot;
  __shared__ double s_tot[2][kWarps];

  if (warp == 0) {
    float p;
    if (a.stats_mode == TP_STATS_EXTERNAL) {
      p = a.mu_hi[c];
    } else {
      const int64_t m = a.nsamp < 64 ? a.nsamp : 64;
      float v = 0.f;
      for (int64_t t = lane; t < m; t += 32) v += load_as_float<DT>(a.x, row + t);
      p = warp_sum_f(v) / (float)m;
    }
    if (lane == 0) s_pivot = p;
  }
  __syncthreads();
  const float p = s_pivot;

  double tot_s = 0.0, tot_q = 0.0;  // lane-0 accumulators of this warp
  for (int k = warp; k < a.nchunk; k += kWarps) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t hi = lo + a.W < a.nsamp ? lo + a.W : a.nsamp;
    double cs = 0.0, cq = 0.0;
    for (int64_t sub = lo; sub < hi; sub += 256) {
      const int64_t sh = sub + 256 < hi ? sub + 256 : hi;
      float fs = 0.f, fq = 0.f;
      for (int64_t t = sub + lane; t < sh; t += 32) {
        const float e = load_as_float<DT>(a.x, row + t) - p;
        fs += e;
        fq += e * e;
      }
      fs = warp_sum_f(fs);
      fq = warp_sum_f(fq);
      cs += (double)fs;
      cq += (double)fq;
    }
    if (lane == 0) {
      chunk_sums[(int64_t)c * a.nchunk + k] = make_double2(cs, cq);
      tot_s += cs;
      tot_q += cq;
    }
  }
  if (lane == 0) {
    s_tot[0][warp] = tot_s;
    s_tot[1][warp] = tot_q;
  }
  __syncthreads();

  // channel statistics; m = mu - p
  __shared__ double s_m, s_sig;
  if (threadIdx.x == 0) {
    double m, sig;
    if (a.stats_mode == TP_STATS_EXTERNAL) {
      m = (double)a.mu_lo[c];
      sig = a.sigma[c];
    } else {
      double S = 0.0, Q = 0.0;
      for (int w = 0; w < kWarps; ++w) {
        S += s_tot[0][w];
        Q += s_tot[1][w];
      }
      const double N = (double)a.nsamp;
      m = S / N;
      double var = Q / N - m * m;
      sig = sqrt(var > 0.0 ? var : 0.0);
      const double mu = (double)p + m;
      a.mu[c] = mu;
      a.sigma[c] = sig;
      const float hi = (float)mu;
      a.mu_hi[c] = hi;
      a.mu_lo[c] = (float)(mu - (double)hi);
      m = mu - (double)p;
    }
    s_m = m;
    s_sig = sig;
  }
  __syncthreads();
  if (!a.enable_channel) return;
  const double m = s_m, tsig = a.tau_c * s_sig;
  for (int k = threadIdx.x; k < a.nchunk; k += kThreads) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t n = (lo + a.W < a.nsamp ? lo + a.W : a.nsamp) - lo;
    const double2 cs = chunk_sums[(int64_t)c * a.nchunk + k];
    const double e = cs.x - (double)n * m;
    a.chunk_raw[(int64_t)c * a.nchunk + k] = (uint8_t)(e > tsig * sqrt((double)n));
  }
}

// Chunk sums (8-bit data), exact.  chunk_sums[c][k] = {sum x, sum x^2}.
__global__ void __launch_bounds__(kThreads) chunk_stats_u8(RfiArgs a, longlong2* chunk_sums) {
  const int c = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)c * a.pitch;
  __shared__ unsigned long long s_tot[2][kWarps];
  unsigned long long tot_s = 0, tot_q = 0;
  for (int k = warp; k < a.nchunk; k += kWarps) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t hi = lo + a.W < a.nsamp ? lo + a.W : a.nsamp;
    unsigned long long s = 0, q = 0;
    for (int64_t t = lo + lane; t < hi; t += 32) {
      const unsigned v = load_u8(a.x, row + t);
      s += v;
      q += v * v;
    }
    s = warp_sum_u64(s);
    q = warp_sum_u64(q);
    if (lane == 0) {
      chunk_sums[(int64_t)c * a.nchunk + k] = make_longlong2((long long)s, (long long)q);
      tot_s += s;
      tot_q += q;
    }
  }
  if (lane == 0) {
    s_tot[0][warp] = tot_s;
    s_tot[1][warp] = tot_q;
  }
  __syncthreads();
  __shared__ long long s_S, s_V;
  __shared__ int s_b;
  if (threadIdx.x == 0) {
    const long long N = a.nsamp;
    if (a.stats_mode == TP_STATS_EXTERNAL) {
      s_b = a.bint[c];
      s_S = 0;
      s_V = 0;
    } else {
      unsigned long long S = 0, Q = 0;
      for (int w = 0; w < kWarps; ++w) {
        S += s_tot[0][w];
        Q += s_tot[1][w];
      }
      const long long V = N * (long long)Q - (long long)S * (long long)S;
      const int b = (int)((2 * (long long)S + N) / (2 * N));
      a.S[c] = (long long)S;
      a.V[c] = V;
      a.bint[c] = b;
      a.mu[c] = __ddiv_rn((double)(long long)S, (double)N);
      a.sigma[c] = __ddiv_rn(__dsqrt_rn((double)V), (double)N);
      s_S = (long long)S;
      s_V = V;
      s_b = b;
    }
  }
  __syncthreads();
  if (!a.enable_channel) return;
  const long long N = a.nsamp, S = s_S, V = s_V, b = s_b;
  const bool ext = a.stats_mode == TP_STATS_EXTERNAL;
  const double tsig = ext ? __dmul_rn(a.tau_c, a.sigma[c]) : 0.0;
  for (int k = threadIdx.x; k < a.nchunk; k += kThreads) {
    const long long lo = (long long)k * a.W;
    const long long n = (lo + a.W < N ? lo + a.W : N) - lo;
    const longlong2 cs = chunk_sums[(int64_t)c * a.nchunk + k];
    bool ex;
    if (ext) {
      const long long e = cs.x - n * b;
      ex = (double)e > __dmul_rn(tsig, __dsqrt_rn((double)n));
    } else {
      const long long e = N * cs.x - n * S;
      ex = (double)e > __dmul_rn(a.tau_c, __dsqrt_rn(__dmul_rn((double)V, (double)n)));
    }
    a.chunk_raw[(int64_t)c * a.nchunk + k] = (uint8_t)ex;
  }
}

// Dilation of the exceedances into flags, per-channel flagged-chunk counts.
// One warp per channel.
__global__ void __launch_bounds__(kThreads) dilate_kernel(RfiArgs a) {
  const int c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.nchan) return;
  const uint8_t* raw = a.chunk_raw;
  const int nk = a.nchunk;
  int cnt = 0;
  for (int k = lane; k < nk; k += 32) {
    const int64_t i = (int64_t)c * nk + k;
    int f = raw[i];
    if (k > 0) f |= raw[i - 1];
    if (k + 1 < nk) f |= raw[i + 1];
    if (a.dilate_channels) {
      if (c > 0) f |= raw[i - nk];
      if (c + 1 < a.nchan) f |= raw[i + nk];
    }
    a.chunk_flag[i] = (uint8_t)(f != 0);
    cnt += f != 0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  if (lane == 0) a.chan_nflag[c] = cnt;
}

// Spectrum threshold (one CTA).  Block statistics: float data sum sigma_c^2 in
// binary64; 8-bit data sum V_c exactly as (V >> 20, V & (2^20 - 1)).  External
// statistics: the threshold was computed on the host and is passed in.
__global__ void __launch_bounds__(kThreads) spectrum_threshold_kernel(RfiArgs a, double ext_thr) {
  __shared__ double s_d[kThreads];
  __shared__ unsigned long long s_hi[kThreads], s_lo[kThreads];
  if (threadIdx.x == 0) *a.spec_nflag = 0;
  if (a.stats_mode == TP_STATS_EXTERNAL) {
    if (threadIdx.x == 0) *a.spec_thr = ext_thr;
    return;
  }
  double v = 0.0;
  unsigned long long hi = 0, lo = 0;
  for (int c = threadIdx.x; c < a.nchan; c += kThreads) {
    if (a.dtype == TP_U8) {
      const unsigned long long V = (unsigned long long)a.V[c];
      hi += V >> 20;
      lo += V & 0xFFFFFull;
    } else {
      v += a.sigma[c] * a.sigma[c];
    }
  }
  s_d[threadIdx.x] = v;
  s_hi[threadIdx.x] = hi;
  s_lo[threadIdx.x] = lo;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_d[threadIdx.x] += s_d[threadIdx.x + o];
      s_hi[threadIdx.x] += s_hi[threadIdx.x + o];
      s_lo[threadIdx.x] += s_lo[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double tot;
    if (a.dtype == TP_U8)
      tot = __dadd_rn(__dmul_rn((double)s_hi[0], 1048576.0), (double)s_lo[0]);
    else
      tot = s_d[0];
    *a.spec_thr = __dmul_rn(a.tau_s, __dsqrt_rn(tot));
  }
}

// Spectrum flags.  CTA = 256 consecutive samples; warp w sums channels
// w, w + 8, ...; lane handles samples t0 + lane + 32 j, j < 8.
template <int DT>
__global__ void __launch_bounds__(kThreads) spectrum_flags_kernel(RfiArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t t0 = (int64_t)blockIdx.x * 256;
  constexpr bool kU8 = DT == TP_U8;
  int kj[8];
  bool vj[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const int64_t t = t0 + lane + 32 * j;
    vj[j] = t < a.nsamp;
    kj[j] = vj[j] ? (int)(t / a.W) : 0;
  }
  __shared__ double s_f[kWarps][256];
  __shared__ long long s_i[kWarps][256];
  if constexpr (!kU8) {
    double acc[8];
    float part[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[j] = 0.0, part[j] = 0.f;
    int n = 0;
    for (int c = warp; c < a.nchan; c += kWarps) {
      const float mh = a.mu_hi[c], ml = a.mu_lo[c];
      const int64_t row = (int64_t)c * a.pitch;
      const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
      const bool any = a.chan_nflag[c] != 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (vj[j] && !(any && cf[kj[j]])) {
          const float v = load_as_float<DT>(a.x, row + t0 + lane + 32 * j);
          part[j] += (v - mh) - ml;
        }
      }
      if (++n == 8) {
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += (double)part[j], part[j] = 0.f;
        n = 0;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) s_f[warp][lane + 32 * j] = acc[j] + (double)part[j];
  } else {
    const bool ext = a.stats_mode == TP_STATS_EXTERNAL;
    const long long N = a.nsamp;
    int sx[8];
    long long sS[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) sx[j] = 0, sS[j] = 0;
    for (int c = warp; c < a.nchan; c += kWarps) {
      const long long off = ext ? (long long)a.bint[c] : a.S[c];
      const int64_t row = (int64_t)c * a.pitch;
      const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
      const bool any = a.chan_nflag[c] != 0;
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (vj[j] && !(any && cf[kj[j]])) {
          sx[j] += (int)load_u8(a.x, row + t0 + lane + 32 * j);
          sS[j] += off;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j)
      s_i[warp][lane + 32 * j] = ext ? (long long)sx[j] - sS[j] : N * (long long)sx[j] - sS[j];
  }
  __syncthreads();
  const int64_t t = t0 + threadIdx.x;
  const double thr = *a.spec_thr;
  bool flag = false;
  if (t < a.nsamp) {
    if (!kU8) {
      double m = 0.0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) m += s_f[w][threadIdx.x];
      flag = m > thr;
    } else {
      long long m = 0;
#pragma unroll
      for (int w = 0; w < kWarps; ++w) m += s_i[w][threadIdx.x];
      flag = (double)m > thr;
    }
  }
  const unsigned bits = __ballot_sync(0xffffffffu, flag);
  if (lane == 0) {
    const int64_t word = (t0 >> 5) + warp;
    if (word * 32 < a.nsamp) a.spec_bits[word] = bits;
    if (bits) atomicAdd(a.spec_nflag, __popc(bits));
  }
}

}  // namespace

cudaError_t launch_rfi(const RfiArgs& a, void* chunk_sums, double ext_thr, cudaStream_t s) {
  if (a.dtype == TP_U8)
    chunk_stats_u8<<<a.nchan, kThreads, 0, s>>>(a, static_cast<longlong2*>(chunk_sums));
  else if (a.dtype == TP_F16)
    chunk_stats_float<TP_F16><<<a.nchan, kThreads, 0, s>>>(a, static_cast<double2*>(chunk_sums));
  else if (a.dtype == TP_BF16)
    chunk_stats_float<TP_BF16><<<a.nchan, kThreads, 0, s>>>(a, static_cast<double2*>(chunk_sums));
  else
    chunk_stats_float<TP_F32><<<a.nchan, kThreads, 0, s>>>(a, static_cast<double2*>(chunk_sums));
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t nflag_bytes = (int64_t)a.nchan * a.nchunk;
  if (a.enable_channel) {
    dilate_kernel<<<(a.nchan + kWarps - 1) / kWarps, kThreads, 0, s>>>(a);
  } else {
    e = cudaMemsetAsync(a.chunk_raw, 0, nflag_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.chunk_flag, 0, nflag_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.chan_nflag, 0, sizeof(int) * a.nchan, s);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  spectrum_threshold_kernel<<<1, kThreads, 0, s>>>(a, ext_thr);
  const int64_t words = (a.nsamp + 31) / 32;
  if (a.enable_spectrum) {
    const unsigned blocks = (unsigned)((a.nsamp + 255) / 256);
    if (a.dtype == TP_U8)
      spectrum_flags_kernel<TP_U8><<<blocks, kThreads, 0, s>>>(a);
    else if (a.dtype == TP_F16)
      spectrum_flags_kernel<TP_F16><<<blocks, kThreads, 0, s>>>(a);
    else if (a.dtype == TP_BF16)
      spectrum_flags_kernel<TP_BF16><<<blocks, kThreads, 0, s>>>(a);
    else
      spectrum_flags_kernel<TP_F32><<<blocks, kThreads, 0, s>>>(a);
  } else {
    e = cudaMemsetAsync(a.spec_bits, 0, sizeof(uint32_t) * words, s);
    if (e != cudaSuccess) return e;
  }
  return cudaGetLastError();
}

}  // namespace tp
