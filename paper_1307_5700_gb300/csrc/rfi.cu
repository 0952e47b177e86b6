// A1-A3: bandpass statistics, channel thresholding and spectrum thresholding
// ("Bandpass Correction", "Channel Thresholding" and "Spectrum Thresholding"
// of Sec. 2.2.1).
//
// Kernel chunk_sums (a CTA per 32 consecutive chunks of one channel): every
// W_c-sample chunk of the window is summed by one warp.  Float data are summed
// as (x - p) with a per-channel pivot p near the mean (the FP32 mean of the
// first 64 samples), in FP32 inside sub-chunks of at most 256 samples and in
// FP64 above that; 8-bit data are summed exactly in integers.  The per-chunk
// sums go to global scratch.  Kernel channel_stats (a warp per channel): the
// channel totals give mu_c and sigma_c, and each chunk is then tested against
// tau_c sigma_c sqrt(n_k).
// Kernel dilate: flag = own exceedance | time neighbours (| channel
// neighbours); per-channel flagged-chunk counts.  Kernel spectrum_threshold
// (a warp per chunk): tau_s sqrt(sum of sigma_c^2 over the channels whose
// chunk is not flagged).  A3 + A4 (one CTA per 32 samples x all channels):
// the sum over channels of the corrected samples of unflagged chunks,
// compared with that threshold, then the staged series with flagged samples
// replaced -- spectrum_substitute_tile / spectrum_substitute_tile_u8 when W_c
// is a multiple of 32 and the channels' parameters fit shared memory,
// spectrum_substitute_kernel otherwise.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>
#include <type_traits>

#include "tp_common.cuh"

namespace tp {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunkBatch = 4;  // W_c = 256 chunks summed per warp and iteration

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

// Power |v|^2 = re^2 + im^2 of a complex voltage sample (int16 real part in
// the low half, imaginary in the high half): exact in 32-bit unsigned
// integers, one rounding to FP32 (none below 2^24).
__device__ __forceinline__ float c16_power(int v) {
  const int re = (short)(v & 0xffff), im = v >> 16;
  return (float)((unsigned)(re * re) + (unsigned)(im * im));
}
template <>
__device__ __forceinline__ float load_as_float<TP_C16>(const void* x, int64_t i) {
  return c16_power(__ldg(static_cast<const int*>(x) + i));
}

// sample formats staged as FP32 y = x - mu (binary32 data, complex-voltage power)
template <int DT>
constexpr bool kStagedF32 = DT == TP_F32 || DT == TP_C16;

// value of 16-bit storage bits (exact in FP32)
template <int DT>
__device__ __forceinline__ float bits_to_float(unsigned short h) {
  if constexpr (DT == TP_F16) {
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
  } else {
    return __uint_as_float((unsigned)h << 16);
  }
}

__device__ __forceinline__ unsigned load_u8(const void* x, int64_t i) {
  return __ldg(static_cast<const unsigned char*>(x) + i);
}

// Nearest value of a 16-bit storage format (ties to even), from the format's
// definition: `sig` significant bits, smallest normal exponent `emin`.
__device__ double round_to_format(double v, int sig, int emin, double maxv) {
  if (v == 0.0 || !isfinite(v)) return v;
  const double a = fabs(v);
  int e;
  frexp(a, &e);
  int qexp = e - sig;
  if (qexp < emin - sig + 1) qexp = emin - sig + 1;
  const double q = ldexp(1.0, qexp);
  double r = rint(a / q) * q;
  if (r > maxv) r = __longlong_as_double(0x7ff0000000000000LL);
  return copysign(r, v);
}

// Bandpass value of a 16-bit format as its bit pattern.
__device__ unsigned short storage_bits(int dtype, double mu) {
  if (dtype == TP_F16) return __half_as_ushort(__double2half(round_to_format(mu, 11, -14, 65504.0)));
  return __bfloat16_as_ushort(__double2bfloat16(round_to_format(mu, 8, -126, 3.3895313892515355e38)));
}

__device__ __forceinline__ double storage_value(int dtype, unsigned short bits) {
  if (dtype == TP_F16) return (double)__half2float(__ushort_as_half(bits));
  return (double)__uint_as_float((unsigned)bits << 16);
}

__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
// (hi, lo) += v: hi takes the FP32 sum, lo its exact rounding error (Knuth's
// two_sum, six FP32 operations; nothing is contracted: --fmad=false)
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float v) {
  const float s = hi + v;
  const float bv = s - hi;
  const float av = s - bv;
  lo += (hi - av) + (v - bv);
  hi = s;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Chunk sums (float data): chunk_sums[c][k] = {sum(x - p), sum((x - p)^2)}
// with p the channel's pivot.  A CTA of chunk_sums_float covers kGroupChunks
// consecutive chunks of one channel (blockIdx.y); when W is a multiple of
// 128 every lane reads float-aligned quads (two per 256-sample sub-chunk).
constexpr int kGroupChunks = kWarps * kChunkBatch;

// four consecutive samples from i (those at or past `lim` read as 0, ok =
// false), converted to FP32 from the storage format
template <int DT>
__device__ __forceinline__ void load4_raw(const void* x, int64_t i, int64_t lim, float (&e)[4], bool (&ok)[4]) {
  if (i + 3 < lim) {
    if constexpr (DT == TP_F32) {
      const float4 v = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(x) + i));
      e[0] = v.x, e[1] = v.y, e[2] = v.z, e[3] = v.w;
    } else if constexpr (DT == TP_C16) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(static_cast<const int*>(x) + i));
      e[0] = c16_power(v.x), e[1] = c16_power(v.y), e[2] = c16_power(v.z), e[3] = c16_power(v.w);
    } else {
      const uint2 v = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(x) + i));
      const unsigned short h[4] = {(unsigned short)(v.x & 0xffff), (unsigned short)(v.x >> 16),
                                   (unsigned short)(v.y & 0xffff), (unsigned short)(v.y >> 16)};
#pragma unroll
      for (int r = 0; r < 4; ++r) e[r] = bits_to_float<DT>(h[r]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) ok[r] = true;
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      ok[r] = i + r < lim;
      e[r] = ok[r] ? load_as_float<DT>(x, i + r) : 0.f;
    }
  }
}

// The channel's pivot (one full warp): the FP32 mean of its first
// min(64, N) samples, or the external mean's high part.  Every kernel that
// needs it recomputes it the same way, so all see the same value.
template <int DT>
__device__ __forceinline__ float channel_pivot(const RfiArgs& a, int c, int lane) {
  if (a.stats_mode == TP_STATS_EXTERNAL) return a.mu_hi[c];
  const int64_t row = (int64_t)c * a.pitch;
  const int64_t m = a.nsamp < 64 ? a.nsamp : 64;
  float v = 0.f;
  for (int64_t t = lane; t < m; t += 32) v += load_as_float<DT>(a.x, row + t);
  return warp_sum_f(v) / (float)m;
}

// the FP32 sums of one <= 256-sample sub-chunk held as two quads per lane
__device__ __forceinline__ float2 quad_sums(const float (&e0)[4], const float (&e1)[4], float p) {
  float fs = 0.f, fq = 0.f;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float d = e0[r] - p;
    fs += d;
    fq += d * d;
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const float d = e1[r] - p;
    fs += d;
    fq += d * d;
  }
  return make_float2(warp_sum_f(fs), warp_sum_f(fq));
}

template <int DT>
__global__ void __launch_bounds__(kThreads) chunk_sums_float(RfiArgs a, double2* chunk_sums) {
  const int c = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)c * a.pitch;
  // every load of the CTA lies in [row, row + nsamp)
  if (!in_bounds(0, a.nsamp, a.pitch, a.status) || !in_bounds(row, a.nsamp, a.x_elems, a.status)) return;
  const int k0 = blockIdx.x * kGroupChunks;
  const int k1 = k0 + kGroupChunks < a.nchunk ? k0 + kGroupChunks : a.nchunk;
  const bool vec = (a.W % 128) == 0;
  // W <= 256: every chunk is one FP32 sub-chunk, its sums stored as float2;
  // wider chunks accumulate their sub-chunks in FP64 (double2)
  const bool single = a.W <= 256;
  float2* sums32 = reinterpret_cast<float2*>(chunk_sums) + (int64_t)c * a.nchunk;
  __shared__ float s_pivot;

  // W = 256: the warp's kChunkBatch full chunks k0 + warp + u kWarps are
  // loaded before the pivot is known (their loads overlap its computation)
  const int nfull = (int)(a.nsamp / 256);
  const bool batch = vec && a.W == 256;
  float e[kChunkBatch][2][4];
  bool ok[kChunkBatch][2][4];
  if (batch) {
#pragma unroll
    for (int u = 0; u < kChunkBatch; ++u) {
      const int k = k0 + warp + u * kWarps;
      if (k < nfull) {
        const int64_t lo = (int64_t)k * 256;
        load4_raw<DT>(a.x, row + lo + 4 * lane, row + lo + 256, e[u][0], ok[u][0]);
        load4_raw<DT>(a.x, row + lo + 128 + 4 * lane, row + lo + 256, e[u][1], ok[u][1]);
      }
    }
  }
  if (warp == 0) {
    const float p = channel_pivot<DT>(a, c, lane);
    if (lane == 0) s_pivot = p;
  }
  __syncthreads();
  const float p = s_pivot;
  if (batch) {
#pragma unroll
    for (int u = 0; u < kChunkBatch; ++u) {
      const int k = k0 + warp + u * kWarps;
      if (k < nfull) {
        const float2 s = quad_sums(e[u][0], e[u][1], p);
        if (lane == 0) sums32[k] = s;
      }
    }
  }
  // the rest: every chunk of the group when W != 256, else a short last chunk
  for (int k = k0 + warp; k < k1; k += kWarps) {
    if (batch && k < nfull) continue;
    const int64_t lo = (int64_t)k * a.W;
    const int64_t hi = lo + a.W < a.nsamp ? lo + a.W : a.nsamp;
    double cs = 0.0, cq = 0.0;
    for (int64_t sub = lo; sub < hi; sub += 256) {
      const int64_t sh = sub + 256 < hi ? sub + 256 : hi;
      float2 s;
      if (vec) {
        float e0[4], e1[4];
        bool q0[4], q1[4];
        load4_raw<DT>(a.x, row + sub + 4 * lane, row + sh, e0, q0);
        load4_raw<DT>(a.x, row + sub + 128 + 4 * lane, row + sh, e1, q1);
        // samples past the end read as p, which adds 0
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          e0[r] = q0[r] ? e0[r] : p;
          e1[r] = q1[r] ? e1[r] : p;
        }
        s = quad_sums(e0, e1, p);
      } else {
        float fs = 0.f, fq = 0.f;
        for (int64_t t = sub + lane; t < sh; t += 32) {
          const float d = load_as_float<DT>(a.x, row + t) - p;
          fs += d;
          fq += d * d;
        }
        s = make_float2(warp_sum_f(fs), warp_sum_f(fq));
      }
      if (single) {
        if (lane == 0) sums32[k] = s;
      } else {
        cs += (double)s.x;
        cq += (double)s.y;
      }
    }
    if (!single && lane == 0) chunk_sums[(int64_t)c * a.nchunk + k] = make_double2(cs, cq);
  }
}

// Channel statistics and chunk exceedances (float data), one warp per
// channel: the binary64 totals of the chunk sums (lane l sums chunks l,
// l + 32, ...; the lanes' totals are combined in a fixed butterfly order),
// mu_c = p + S / N and sigma_c = sqrt(Q / N - (S / N)^2); chunk k exceeds when
// sum(x - mu_c) > tau_c sigma_c sqrt(n_k).
template <int DT>
__global__ void __launch_bounds__(kThreads) channel_stats_float(RfiArgs a, const double2* chunk_sums) {
  const int c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.nchan) return;
  const float p = channel_pivot<DT>(a, c, lane);
  const bool single = a.W <= 256;
  const float2* sums32 = reinterpret_cast<const float2*>(chunk_sums) + (int64_t)c * a.nchunk;
  auto chunk_sum = [&](int k) -> double2 {
    if (single) {
      const float2 f = sums32[k];
      return make_double2((double)f.x, (double)f.y);
    }
    return chunk_sums[(int64_t)c * a.nchunk + k];
  };
  double m, sig;
  if (a.stats_mode == TP_STATS_EXTERNAL) {
    m = (double)a.mu_lo[c];
    sig = a.sigma[c];
  } else {
    double S = 0.0, Q = 0.0;
    if (single) {
      // FP32 chunk sums: totals carried as exact FP32 pairs (two_sum), the
      // lanes' pairs combined in a fixed butterfly order
      float sh = 0.f, sl = 0.f, qh = 0.f, ql = 0.f;
      for (int k = lane; k < a.nchunk; k += 32) {
        const float2 v = sums32[k];
        two_sum_acc(sh, sl, v.x);
        two_sum_acc(qh, ql, v.y);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const float osh = __shfl_xor_sync(0xffffffffu, sh, o), osl = __shfl_xor_sync(0xffffffffu, sl, o);
        const float oqh = __shfl_xor_sync(0xffffffffu, qh, o), oql = __shfl_xor_sync(0xffffffffu, ql, o);
        two_sum_acc(sh, sl, osh);
        sl += osl;
        two_sum_acc(qh, ql, oqh);
        ql += oql;
      }
      S = (double)sh + (double)sl;
      Q = (double)qh + (double)ql;
    } else {
      for (int k = lane; k < a.nchunk; k += 32) {
        const double2 v = chunk_sum(k);
        S += v.x;
        Q += v.y;
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        S += __shfl_xor_sync(0xffffffffu, S, o);
        Q += __shfl_xor_sync(0xffffffffu, Q, o);
      }
    }
    const double N = (double)a.nsamp;
    m = S / N;
    const double var = Q / N - m * m;
    sig = sqrt(var > 0.0 ? var : 0.0);
    const double mu = (double)p + m;
    if (lane == 0) {
      a.mu[c] = mu;
      a.sigma[c] = sig;
      const float hi = (float)mu;
      a.mu_hi[c] = hi;
      a.mu_lo[c] = (float)(mu - (double)hi);
      if (DT == TP_F16 || DT == TP_BF16) a.b16[c] = storage_bits(DT, mu);
    }
    m = mu - (double)p;
  }
  if (lane == 0 && (a.fit || a.run)) a.pivot[c] = p;
  // with the fitted bandpass the chunk test waits for the fit
  // (fit_chunk_test), with running statistics for their update
  // (running_chunk_test)
  if (!a.enable_channel || a.fit || a.run) return;
  const double tsig = a.tau_c * sig;
  const double thr_w = tsig * sqrt((double)a.W);  // the threshold of a full chunk
  // full chunks with FP32 sums are first tested in FP32: e32 - thr32 is
  // within 2^-23 (|s_k| + |W m| + |thr|) of the binary64 e - thr, so outside
  // a guard band eight times wider the FP32 sign is the binary64 decision;
  // inside it (and for non-finite values) the binary64 test decides
  const float thr32 = (float)thr_w, nm32 = (float)((double)a.W * m);
  for (int k = lane; k < a.nchunk; k += 32) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t n = (lo + a.W < a.nsamp ? lo + a.W : a.nsamp) - lo;
    int ex = 2;
    if (single && n == a.W) {
      const float cx = sums32[k].x;
      const float d = (cx - nm32) - thr32;
      const float guard = 9.5367431640625e-7f * (fabsf(cx) + fabsf(nm32) + fabsf(thr32));
      ex = d > guard ? 1 : (-d > guard ? 0 : 2);
    }
    if (ex == 2) {
      const double2 cs = chunk_sum(k);
      const double e = cs.x - (double)n * m;
      ex = e > (n == a.W ? thr_w : tsig * sqrt((double)n)) ? 1 : 0;
    }
    a.chunk_raw[(int64_t)c * a.nchunk + k] = (uint8_t)ex;
  }
}

// Chunk sums (8-bit data), exact: chunk_sums[c][k] = {sum x, sum x^2}.  A CTA
// of chunk_sums_u8 covers kGroupChunks consecutive chunks of one channel
// (blockIdx.y).  With W = 256 and 8-byte aligned rows each lane reads 8
// samples of a chunk with one load and sums them with byte dot products.
__global__ void __launch_bounds__(kThreads) chunk_sums_u8(RfiArgs a, longlong2* chunk_sums) {
  const int c = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t row = (int64_t)c * a.pitch;
  // every load of the CTA lies in [row, row + nsamp)
  if (!in_bounds(0, a.nsamp, a.pitch, a.status) || !in_bounds(row, a.nsamp, a.x_elems, a.status)) return;
  const int k0 = blockIdx.x * kGroupChunks;
  const int k1 = k0 + kGroupChunks < a.nchunk ? k0 + kGroupChunks : a.nchunk;
  const unsigned char* xr = static_cast<const unsigned char*>(a.x) + row;
  const int nfull = (int)(a.nsamp / 256);
  const bool batch = a.W == 256 && ((reinterpret_cast<uintptr_t>(xr)) & 7) == 0;
  if (batch) {
    uint2 w[kChunkBatch];
#pragma unroll
    for (int u = 0; u < kChunkBatch; ++u) {
      const int k = k0 + warp + u * kWarps;
      w[u] = k < nfull ? __ldg(reinterpret_cast<const uint2*>(xr + (int64_t)k * 256) + lane) : make_uint2(0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < kChunkBatch; ++u) {
      const int k = k0 + warp + u * kWarps;
      if (k >= nfull) continue;
      // sum x <= 256 x 255 and sum x^2 <= 256 x 255^2 fit 32 bits
      unsigned s = __dp4a(w[u].x, 0x01010101u, 0u);
      s = __dp4a(w[u].y, 0x01010101u, s);
      unsigned q = __dp4a(w[u].x, w[u].x, 0u);
      q = __dp4a(w[u].y, w[u].y, q);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xffffffffu, s, o);
        q += __shfl_xor_sync(0xffffffffu, q, o);
      }
      if (lane == 0) chunk_sums[(int64_t)c * a.nchunk + k] = make_longlong2((long long)s, (long long)q);
    }
  }
  for (int k = k0 + warp; k < k1; k += kWarps) {
    if (batch && k < nfull) continue;
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
    if (lane == 0) chunk_sums[(int64_t)c * a.nchunk + k] = make_longlong2((long long)s, (long long)q);
  }
}

// Channel statistics and chunk exceedances (8-bit data), one warp per channel,
// in exact integers: S = sum x, V = N sum x^2 - S^2, b_c = floor(S / N + 1/2);
// chunk k exceeds when N s_k - n_k S > tau_c sqrt(V n_k) (block statistics;
// s_k - n_k b_c > tau_c sigma_c sqrt(n_k) with external ones).  The binary64
// threshold of a full chunk is computed once; an exact integer e exceeds it
// exactly when it exceeds the threshold's floor.
__global__ void __launch_bounds__(kThreads) channel_stats_u8(RfiArgs a, const longlong2* chunk_sums) {
  const int c = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (c >= a.nchan) return;
  const long long N = a.nsamp;
  const longlong2* cs_row = chunk_sums + (int64_t)c * a.nchunk;
  const bool ext = a.stats_mode == TP_STATS_EXTERNAL;
  long long S = 0, V = 0, b;
  if (ext) {
    b = a.bint[c];
  } else {
    unsigned long long s = 0, q = 0;
    for (int k = lane; k < a.nchunk; k += 32) {
      const longlong2 v = cs_row[k];
      s += (unsigned long long)v.x;
      q += (unsigned long long)v.y;
    }
    s = warp_sum_u64(s);
    q = warp_sum_u64(q);
    S = (long long)s;
    V = N * (long long)q - S * S;
    b = (2 * S + N) / (2 * N);
    if (lane == 0) {
      a.S[c] = S;
      a.V[c] = V;
      a.bint[c] = (int)b;
      a.mu[c] = __ddiv_rn((double)S, (double)N);
      a.sigma[c] = __ddiv_rn(__dsqrt_rn((double)V), (double)N);
    }
  }
  if (!a.enable_channel || a.fit || a.run) return;
  const double tsig = ext ? __dmul_rn(a.tau_c, a.sigma[c]) : 0.0;
  auto threshold = [&](long long n) -> double {
    return ext ? __dmul_rn(tsig, __dsqrt_rn((double)n))
               : __dmul_rn(a.tau_c, __dsqrt_rn(__dmul_rn((double)V, (double)n)));
  };
  const double thr_w = threshold(a.W);
  // |e| <= 255 N W keeps (double)e exact below 2^53; the integer comparison
  // then decides as the binary64 one does
  const bool int_cmp = isfinite(thr_w) && fabs(thr_w) < 4.0e18 && 255.0 * (double)N * (double)a.W < 9.0e15;
  const long long e_w = int_cmp ? (long long)floor(thr_w) : 0;
  for (int k = lane; k < a.nchunk; k += 32) {
    const long long lo = (long long)k * a.W;
    const long long n = (lo + a.W < N ? lo + a.W : N) - lo;
    const longlong2 cs = cs_row[k];
    const long long e = ext ? cs.x - n * b : N * cs.x - n * S;
    bool ex;
    if (n == a.W && int_cmp)
      ex = e > e_w;
    else
      ex = (double)e > (n == a.W ? thr_w : threshold(n));
    a.chunk_raw[(int64_t)c * a.nchunk + k] = (uint8_t)ex;
  }
}

// Launch of the A1-A2 statistics kernels on the window described by a.
template <int DT>
cudaError_t launch_stats_float(const RfiArgs& a, void* chunk_sums, cudaStream_t s) {
  const dim3 grid((unsigned)((a.nchunk + kGroupChunks - 1) / kGroupChunks), (unsigned)a.nchan);
  chunk_sums_float<DT><<<grid, kThreads, 0, s>>>(a, static_cast<double2*>(chunk_sums));
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  channel_stats_float<DT><<<(unsigned)((a.nchan + kWarps - 1) / kWarps), kThreads, 0, s>>>(
      a, static_cast<const double2*>(chunk_sums));
  return cudaGetLastError();
}

cudaError_t launch_stats(const RfiArgs& a, void* chunk_sums, cudaStream_t s) {
  if (a.dtype == TP_U8) {
    const dim3 grid((unsigned)((a.nchunk + kGroupChunks - 1) / kGroupChunks), (unsigned)a.nchan);
    chunk_sums_u8<<<grid, kThreads, 0, s>>>(a, static_cast<longlong2*>(chunk_sums));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    channel_stats_u8<<<(unsigned)((a.nchan + kWarps - 1) / kWarps), kThreads, 0, s>>>(
        a, static_cast<const longlong2*>(chunk_sums));
    return cudaGetLastError();
  }
  if (a.dtype == TP_F16) return launch_stats_float<TP_F16>(a, chunk_sums, s);
  if (a.dtype == TP_BF16) return launch_stats_float<TP_BF16>(a, chunk_sums, s);
  if (a.dtype == TP_C16) return launch_stats_float<TP_C16>(a, chunk_sums, s);
  return launch_stats_float<TP_F32>(a, chunk_sums, s);
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

// Spectrum thresholds, one per chunk k (reading R6): tau_s times the square
// root of the sum of the spreads of the channels whose chunk k is not flagged.
// Every CTA sums the spreads of all channels (binary64 sigma_c^2 in a fixed
// tree order; 8-bit block statistics: the exact integers V_c, kept as
// (V >> 20, V & (2^20 - 1))), then one warp per chunk subtracts the sum over
// the few channels flagged in it.  CTA 0 also sums the bandpass values
// (16-bit and 8-bit staging subtract that sum once).
__global__ void __launch_bounds__(kThreads) spectrum_threshold_kernel(RfiArgs a) {
  __shared__ double s_d[kThreads];
  __shared__ unsigned long long s_hi[kThreads], s_lo[kThreads];
  // exact integer spreads: 8-bit data with the block's own statistics
  const bool exact = a.dtype == TP_U8 && !a.fit && !a.run && a.stats_mode != TP_STATS_EXTERNAL;
  if (blockIdx.x == 0) {
    if (threadIdx.x == 0) *a.spec_nflag = 0;
    double bs = 0.0;
    if (a.dtype == TP_U8 || a.dtype == TP_F16 || a.dtype == TP_BF16)
      for (int c = threadIdx.x; c < a.nchan; c += kThreads)
        bs += a.dtype == TP_U8 ? (double)a.bint[c] : storage_value(a.dtype, a.b16[c]);
    s_d[threadIdx.x] = bs;
    __syncthreads();
    for (int o = kThreads / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) s_d[threadIdx.x] += s_d[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) *a.bsum = s_d[0];
    __syncthreads();
  }
  double v = 0.0;
  unsigned long long hi = 0, lo = 0;
  for (int c = threadIdx.x; c < a.nchan; c += kThreads) {
    if (exact) {
      const unsigned long long V = (unsigned long long)a.V[c];
      hi += V >> 20;
      lo += V & 0xFFFFFull;
    } else {
      v = __dadd_rn(v, __dmul_rn(a.sigma[c], a.sigma[c]));
    }
  }
  s_d[threadIdx.x] = v;
  s_hi[threadIdx.x] = hi;
  s_lo[threadIdx.x] = lo;
  __syncthreads();
  for (int o = kThreads / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_d[threadIdx.x] = __dadd_rn(s_d[threadIdx.x], s_d[threadIdx.x + o]);
      s_hi[threadIdx.x] += s_hi[threadIdx.x + o];
      s_lo[threadIdx.x] += s_lo[threadIdx.x + o];
    }
    __syncthreads();
  }
  const int k = blockIdx.x * kWarps + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (k >= a.nchunk) return;
  double fv = 0.0;
  unsigned long long fhi = 0, flo = 0;
  // the lane's channels c = lane, lane + 32, ... in order, eight at a time
  // (their flag loads issued together)
  for (int c0 = lane; c0 < a.nchan; c0 += 32 * 8) {
    int nf[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) nf[u] = c0 + 32 * u < a.nchan ? a.chan_nflag[c0 + 32 * u] : 0;
    bool fl[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) fl[u] = nf[u] != 0 && a.chunk_flag[(int64_t)(c0 + 32 * u) * a.nchunk + k];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      if (!fl[u]) continue;
      const int c = c0 + 32 * u;
      if (exact) {
        const unsigned long long V = (unsigned long long)a.V[c];
        fhi += V >> 20;
        flo += V & 0xFFFFFull;
      } else {
        fv = __dadd_rn(fv, __dmul_rn(a.sigma[c], a.sigma[c]));
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    fv = __dadd_rn(fv, __shfl_xor_sync(0xffffffffu, fv, o));
    fhi += __shfl_xor_sync(0xffffffffu, fhi, o);
    flo += __shfl_xor_sync(0xffffffffu, flo, o);
  }
  if (lane == 0) {
    double tot;
    if (exact) {
      // the unflagged channels' sum, exactly: the flagged parts are sub-sums
      tot = __dadd_rn(__dmul_rn((double)(s_hi[0] - fhi), 1048576.0), (double)(s_lo[0] - flo));
    } else {
      tot = __dadd_rn(s_d[0], -fv);
      tot = tot > 0.0 ? tot : 0.0;
    }
    a.spec_thr[k] = __dmul_rn(a.tau_s, __dsqrt_rn(tot));
  }
}

// A3 + A4: spectrum flags and the substituted, bandpass-corrected series
//   y[c][t] = 0 if chunk (c, t / W) or spectrum t is flagged, else x - b_c
// (float data: (x - mu_hi) - mu_lo in FP32; 8-bit data: the exact integer
// x - b_c, stored as FP32).  CTA = 32 consecutive samples (one flag word) x
// every channel; thread (g = tid / 8, q = tid % 8) handles samples
// t0 + 4q .. t0 + 4q + 3 of channels g, g + 32, ...  Pass 1 sums the corrected
// samples of unflagged chunks over channels (FP32 runs of 8 channels folded
// into FP64; exact integers for 8-bit data); pass 2 re-reads the tile (an L2
// hit) and writes y.
template <int DT>
__device__ __forceinline__ void load_quad(const void* x, int64_t i, int64_t valid, float (&v)[4]) {
  if (valid >= 4) {
    if constexpr (DT == TP_F32) {
      const float4 f = __ldg(reinterpret_cast<const float4*>(static_cast<const float*>(x) + i));
      v[0] = f.x, v[1] = f.y, v[2] = f.z, v[3] = f.w;
    } else if constexpr (DT == TP_C16) {
      const int4 f = __ldg(reinterpret_cast<const int4*>(static_cast<const int*>(x) + i));
      v[0] = c16_power(f.x), v[1] = c16_power(f.y), v[2] = c16_power(f.z), v[3] = c16_power(f.w);
    } else if constexpr (DT == TP_U8) {
      const unsigned w = __ldg(reinterpret_cast<const unsigned*>(static_cast<const unsigned char*>(x) + i));
#pragma unroll
      for (int r = 0; r < 4; ++r) v[r] = (float)((w >> (8 * r)) & 0xffu);
    } else {
      const uint2 u = __ldg(reinterpret_cast<const uint2*>(static_cast<const unsigned short*>(x) + i));
      const unsigned short h[4] = {(unsigned short)(u.x & 0xffff), (unsigned short)(u.x >> 16),
                                   (unsigned short)(u.y & 0xffff), (unsigned short)(u.y >> 16)};
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if constexpr (DT == TP_F16)
          asm("cvt.f32.f16 %0, %1;" : "=f"(v[r]) : "h"(h[r]));
        else
          v[r] = __uint_as_float((unsigned)h[r] << 16);
      }
    }
  } else {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (r < valid) {
        if constexpr (DT == TP_U8)
          v[r] = (float)load_u8(x, i + r);
        else
          v[r] = load_as_float<DT>(x, i + r);
      } else {
        v[r] = 0.f;
      }
    }
  }
}

// Stores staged FP32 values o[0 .. n) of channel c, samples tq .. tq + n - 1
// (a float4 for a full quad).
__device__ __forceinline__ void store_staged_f32(void* yv, int64_t ypitch, int c, int64_t tq, const float (&o)[4],
                                                 int n) {
  float* dst = static_cast<float*>(yv) + (int64_t)c * ypitch + tq;
  if (n == 4) {
    *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
  } else {
    for (int r = 0; r < n; ++r) dst[r] = o[r];
  }
}

template <int DT>
__global__ void __launch_bounds__(kThreads) spectrum_substitute_kernel(RfiArgs a, void* __restrict__ yv,
                                                                       int64_t ypitch) {
  constexpr bool kU8 = DT == TP_U8;
  const int tid = threadIdx.x;
  const int g = tid >> 3, q = tid & 7;
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t tq = t0 + 4 * q;
  const int64_t left = a.nsamp - tq;
  const int valid = left >= 4 ? 4 : (left > 0 ? (int)left : 0);
  // chunk index of each sample (one division when the CTA's 32 samples lie
  // in one chunk)
  int kk[4];
  {
    const int k0 = (int)(t0 / a.W);
    const bool one = (int64_t)(k0 + 1) * a.W >= t0 + 32;
#pragma unroll
    for (int r = 0; r < 4; ++r) kk[r] = r < valid ? (one ? k0 : (int)((tq + r) / a.W)) : 0;
  }
  __shared__ float s_fh[32][33], s_fl[32][33];
  __shared__ long long s_i[32][33];
  __shared__ unsigned s_word;

  if (a.enable_spectrum) {
    if constexpr (!kU8) {
      // (hi, lo): an unevaluated FP32 pair, the running sum of the groups'
      // partial sums carried without rounding error (two_sum)
      float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
      float part[4] = {0.f, 0.f, 0.f, 0.f};
      // channels g, g + 32, ... in groups of 8: the group's loads are issued
      // together, its FP32 partial sums added to (hi, lo) after the group
      for (int c0 = g; c0 < a.nchan; c0 += 32 * 8) {
        float v[8][4];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + 32 * u;
          if (c < a.nchan) {
            if (in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status))
              load_quad<DT>(a.x, (int64_t)c * a.pitch + tq, valid, v[u]);
            else
              v[u][0] = v[u][1] = v[u][2] = v[u][3] = 0.f;
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int c = c0 + 32 * u;
          if (c >= a.nchan) break;
          const float mh = a.mu_hi[c], ml = a.mu_lo[c];
          const bool any = a.chan_nflag[c] != 0;
          const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r < valid && !(any && cf[kk[r]])) part[r] += (v[u][r] - mh) - ml;
        }
        if (c0 + 32 * 7 < a.nchan) {
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            two_sum_acc(hi[r], lo[r], part[r]);
            part[r] = 0.f;
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        two_sum_acc(hi[r], lo[r], part[r]);
        s_fh[g][4 * q + r] = hi[r];
        s_fl[g][4 * q + r] = lo[r];
      }
    } else {
      // external or fitted bandpass: sums of x - b_c (integer b_c)
      const bool ext = a.stats_mode == TP_STATS_EXTERNAL || a.fit || a.run;
      int sx[4] = {0, 0, 0, 0};
      long long sS[4] = {0, 0, 0, 0};
      for (int c = g; c < a.nchan; c += 32) {
        float v[4] = {0.f, 0.f, 0.f, 0.f};
        if (in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status))
          load_quad<DT>(a.x, (int64_t)c * a.pitch + tq, valid, v);
        const long long off = ext ? (long long)a.bint[c] : a.S[c];
        const bool any = a.chan_nflag[c] != 0;
        const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < valid && !(any && cf[kk[r]])) {
            sx[r] += (int)v[r];
            sS[r] += off;
          }
      }
      const long long N = a.nsamp;
#pragma unroll
      for (int r = 0; r < 4; ++r) s_i[g][4 * q + r] = ext ? (long long)sx[r] - sS[r] : N * (long long)sx[r] - sS[r];
    }
    __syncthreads();
    if (tid < 32) {
      bool flag = false;
      if (t0 + tid < a.nsamp) {
        const double thr = a.spec_thr[(t0 + tid) / a.W];
        if constexpr (!kU8) {
          float mh = 0.f, ml = 0.f;
          for (int w = 0; w < 32; ++w) {
            two_sum_acc(mh, ml, s_fh[w][tid]);
            ml += s_fl[w][tid];
          }
          flag = (double)mh + (double)ml > thr;
        } else {
          long long m = 0;
          for (int w = 0; w < 32; ++w) m += s_i[w][tid];
          flag = (double)m > thr;
        }
      }
      const unsigned bits = __ballot_sync(0xffffffffu, flag);
      if (tid == 0) {
        s_word = bits;
        if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = bits;
        if (bits) atomicAdd(a.spec_nflag, __popc(bits));
      }
    }
  } else if (tid == 0) {
    s_word = 0u;
    if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = 0u;
  }
  __syncthreads();
  const unsigned word = s_word;
  bool sflag[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) sflag[r] = (word >> (4 * q + r)) & 1u;

  // pass 2: y (FP32 data: x - mu, flagged -> 0) or the stored samples x~
  // (16-bit data: flagged -> b16; 8-bit data: flagged -> b, widened to 16-bit
  // integers)
  if (valid == 0) return;
  if (valid == 4) {
    // full 4-sample quads: raw loads of 8 channels (c, c + 32, ..., c + 224)
    // issued together, then substitution and stores
    using Raw = typename std::conditional<
        DT == TP_F32, float4,
        typename std::conditional<DT == TP_C16, int4,
                                  typename std::conditional<DT == TP_U8, unsigned, uint2>::type>::type>::type;
    constexpr int kU = 8;
    for (int c0 = g; c0 < a.nchan; c0 += 32 * kU) {
      Raw raw[kU];
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int c = c0 + 32 * u;
        if (c < a.nchan) {
          if (in_bounds((int64_t)c * a.pitch + tq, 4, a.x_elems, a.status))
            raw[u] = __ldg(reinterpret_cast<const Raw*>(static_cast<const char*>(a.x) +
                                                        ((int64_t)c * a.pitch + tq) * sizeof(Raw) / 4));
          else
            raw[u] = Raw{};
        }
      }
#pragma unroll
      for (int u = 0; u < kU; ++u) {
        const int c = c0 + 32 * u;
        if (c >= a.nchan) break;
        if (!in_bounds((int64_t)c * ypitch + tq, 4, a.y_elems, a.status)) continue;
        const bool any = a.chan_nflag[c] != 0;
        const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
        bool fl[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) fl[r] = sflag[r] || (any && cf[kk[r]]);
        if constexpr (kStagedF32<DT>) {
          float v[4];
          if constexpr (DT == TP_C16)
            v[0] = c16_power(raw[u].x), v[1] = c16_power(raw[u].y), v[2] = c16_power(raw[u].z),
            v[3] = c16_power(raw[u].w);
          else
            v[0] = raw[u].x, v[1] = raw[u].y, v[2] = raw[u].z, v[3] = raw[u].w;
          const float mh = a.mu_hi[c], ml = a.mu_lo[c];
          float o[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) o[r] = fl[r] ? 0.f : (v[r] - mh) - ml;
          store_staged_f32(yv, ypitch, c, tq, o, 4);
        } else if constexpr (DT == TP_U8) {
          const unsigned b = (unsigned)a.bint[c];
          unsigned h[4];
#pragma unroll
          for (int r = 0; r < 4; ++r) h[r] = fl[r] ? b : ((raw[u] >> (8 * r)) & 0xffu);
          *reinterpret_cast<uint2*>(static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq) =
              make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
        } else {
          const unsigned short b = a.b16[c];
          unsigned short h[4] = {(unsigned short)(raw[u].x & 0xffff), (unsigned short)(raw[u].x >> 16),
                                 (unsigned short)(raw[u].y & 0xffff), (unsigned short)(raw[u].y >> 16)};
#pragma unroll
          for (int r = 0; r < 4; ++r) h[r] = fl[r] ? b : h[r];
          if (a.stage_f32) {
            // FP32 staging (for the FP32 kernel shapes): y = x~ - b, one
            // rounding of the difference of two exactly converted stored
            // values; flagged samples give exactly 0
            const float bf = bits_to_float<DT>(b);
            const float o[4] = {bits_to_float<DT>(h[0]) - bf, bits_to_float<DT>(h[1]) - bf,
                                bits_to_float<DT>(h[2]) - bf, bits_to_float<DT>(h[3]) - bf};
            store_staged_f32(yv, ypitch, c, tq, o, 4);
          } else {
            *reinterpret_cast<uint2*>(static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq) =
                make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16), (unsigned)h[2] | ((unsigned)h[3] << 16));
          }
        }
      }
    }
    return;
  }
  // the window's last, partial quad
  for (int c = g; c < a.nchan; c += 32) {
    if (!in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status) ||
        !in_bounds((int64_t)c * ypitch + tq, valid, a.y_elems, a.status))
      continue;
    const bool any = a.chan_nflag[c] != 0;
    const uint8_t* cf = a.chunk_flag + (int64_t)c * a.nchunk;
    bool fl[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) fl[r] = sflag[r] || (any && cf[kk[r]]);
    if constexpr (kStagedF32<DT>) {
      float v[4];
      load_quad<DT>(a.x, (int64_t)c * a.pitch + tq, valid, v);
      const float mh = a.mu_hi[c], ml = a.mu_lo[c];
      float o[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) o[r] = fl[r] ? 0.f : (v[r] - mh) - ml;
      store_staged_f32(yv, ypitch, c, tq, o, valid);
    } else if constexpr (DT == TP_U8) {
      // 8-bit data: x~ (flagged -> b) widened to 16-bit integers
      const uint8_t* src = static_cast<const uint8_t*>(a.x) + (int64_t)c * a.pitch + tq;
      const unsigned b = (unsigned)a.bint[c];
      unsigned short* dst = static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq;
      unsigned h[4];
      if (valid == 4) {
        const unsigned u = __ldg(reinterpret_cast<const unsigned*>(src));
#pragma unroll
        for (int r = 0; r < 4; ++r) h[r] = fl[r] ? b : ((u >> (8 * r)) & 0xffu);
        *reinterpret_cast<uint2*>(dst) = make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16));
      } else {
        for (int r = 0; r < valid; ++r) dst[r] = (unsigned short)(fl[r] ? b : __ldg(src + r));
      }
    } else {
      unsigned short h[4];
      {
        const unsigned short* src = static_cast<const unsigned short*>(a.x) + (int64_t)c * a.pitch + tq;
        const unsigned short b = a.b16[c];
        if (valid == 4) {
          const uint2 u = __ldg(reinterpret_cast<const uint2*>(src));
          h[0] = u.x & 0xffff, h[1] = u.x >> 16, h[2] = u.y & 0xffff, h[3] = u.y >> 16;
        } else {
#pragma unroll
          for (int r = 0; r < 4; ++r) h[r] = r < valid ? __ldg(src + r) : 0;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) h[r] = fl[r] ? b : h[r];
      }
      if (a.stage_f32) {
        // FP32 staging (for the FP32 kernel shapes): y = x~ - b, one rounding
        // of the difference of two exactly converted stored values; flagged
        // samples give exactly 0
        const float bf = bits_to_float<DT>(a.b16[c]);
        float o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) o[r] = bits_to_float<DT>(h[r]) - bf;
        store_staged_f32(yv, ypitch, c, tq, o, valid);
        continue;
      }
      unsigned short* dst = static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq;
      if (valid == 4) {
        *reinterpret_cast<uint2*>(dst) = make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16),
                                                    (unsigned)h[2] | ((unsigned)h[3] << 16));
      } else {
        for (int r = 0; r < valid; ++r) dst[r] = h[r];
      }
    }
  }
}

// L2 eviction-priority policies and hinted 16- / 8-byte global accesses: the
// spectrum stage reads its tile twice (pass 1, then pass 2 right after the
// flags are known) and writes the staged series once; the first read keeps
// its lines (evict_last), the re-read and the staged stores mark theirs as
// the first to go (evict_first), so that the writes do not push the tile
// out of L2 before its re-read.
__device__ __forceinline__ uint64_t l2_policy(bool keep) {
  uint64_t pol;
  if (keep)
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  else
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ uint4 ld_hint16(const void* p, uint64_t pol) {
  uint4 v;
  asm volatile("ld.global.nc.L2::cache_hint.v4.u32 {%0, %1, %2, %3}, [%4], %5;"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ uint2 ld_hint8(const void* p, uint64_t pol) {
  uint2 v;
  asm volatile("ld.global.nc.L2::cache_hint.v2.u32 {%0, %1}, [%2], %3;" : "=r"(v.x), "=r"(v.y) : "l"(p), "l"(pol));
  return v;
}
__device__ __forceinline__ void st_hint16(void* p, uint4 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v4.u32 [%0], {%1, %2, %3, %4}, %5;" ::"l"(p), "r"(v.x), "r"(v.y), "r"(v.z),
               "r"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_hint8(void* p, uint2 v, uint64_t pol) {
  asm volatile("st.global.L2::cache_hint.v2.u32 [%0], {%1, %2}, %3;" ::"l"(p), "r"(v.x), "r"(v.y), "l"(pol) : "memory");
}

// store_staged_f32 with the stores' L2 policy pol
__device__ __forceinline__ void store_staged_f32_hint(void* yv, int64_t ypitch, int c, int64_t tq,
                                                      const float (&o)[4], int n, uint64_t pol) {
  float* dst = static_cast<float*>(yv) + (int64_t)c * ypitch + tq;
  if (n == 4) {
    st_hint16(dst, make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]), __float_as_uint(o[3])),
              pol);
  } else {
    for (int r = 0; r < n; ++r) dst[r] = o[r];
  }
}

// The raw 4-sample quad at element i of a float-data window (16 bytes of
// FP32 or complex int16 samples, 8 bytes of 16-bit samples), with policy pol.
template <int DT>
__device__ __forceinline__ uint4 ld_raw_quad(const void* x, int64_t i, uint64_t pol) {
  if constexpr (DT == TP_F32 || DT == TP_C16) {
    return ld_hint16(static_cast<const uint32_t*>(x) + i, pol);
  } else {
    const uint2 u = ld_hint8(static_cast<const unsigned short*>(x) + i, pol);
    return make_uint4(u.x, u.y, 0u, 0u);
  }
}

// FP32 values of a raw quad (ld_raw_quad)
template <int DT>
__device__ __forceinline__ void raw_quad_values(uint4 u, float (&v)[4]) {
  if constexpr (DT == TP_F32) {
    v[0] = __uint_as_float(u.x), v[1] = __uint_as_float(u.y), v[2] = __uint_as_float(u.z), v[3] = __uint_as_float(u.w);
  } else if constexpr (DT == TP_C16) {
    v[0] = c16_power((int)u.x), v[1] = c16_power((int)u.y), v[2] = c16_power((int)u.z), v[3] = c16_power((int)u.w);
  } else {
    v[0] = bits_to_float<DT>((unsigned short)(u.x & 0xffff)), v[1] = bits_to_float<DT>((unsigned short)(u.x >> 16));
    v[2] = bits_to_float<DT>((unsigned short)(u.y & 0xffff)), v[3] = bits_to_float<DT>((unsigned short)(u.y >> 16));
  }
}

// A3 + A4 for float data when each CTA's 32 samples lie in one chunk (W a
// multiple of 32) and the channels' parameters fit shared memory: the same
// arithmetic as spectrum_substitute_kernel, in the same order (so the same
// flags and the same staged values), with every channel's (mu_hi, mu_lo),
// chunk flag for the CTA's chunk and 16-bit bandpass value read once per CTA
// into shared memory instead of once per channel and pass by every thread.
constexpr int kTileMaxChannels = 4096;

template <int DT>
__global__ void __launch_bounds__(kThreads) spectrum_substitute_tile(RfiArgs a, void* __restrict__ yv,
                                                                     int64_t ypitch) {
  static_assert(DT != TP_U8, "float data");
  extern __shared__ __align__(16) unsigned char s_dyn[];
  float2* s_mu = reinterpret_cast<float2*>(s_dyn);                            // [nchan] (mu_hi, mu_lo)
  unsigned short* s_b16 = reinterpret_cast<unsigned short*>(s_mu + a.nchan);  // [nchan] (16-bit data)
  uint8_t* s_cf = reinterpret_cast<uint8_t*>(s_b16 + a.nchan);                // [nchan] chunk flag
  __shared__ float s_fh[32][33], s_fl[32][33];
  __shared__ unsigned s_word;
  const int tid = threadIdx.x;
  const int g = tid >> 3, q = tid & 7;
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t tq = t0 + 4 * q;
  const int64_t left = a.nsamp - tq;
  const int valid = left >= 4 ? 4 : (left > 0 ? (int)left : 0);
  const int k = (int)(t0 / a.W);
  const uint64_t keep = l2_policy(true), drop = l2_policy(false);
  for (int c = tid; c < a.nchan; c += kThreads) {
    s_mu[c] = make_float2(a.mu_hi[c], a.mu_lo[c]);
    if constexpr (DT == TP_F16 || DT == TP_BF16) s_b16[c] = a.b16[c];
    s_cf[c] = (uint8_t)(a.chan_nflag[c] != 0 && a.chunk_flag[(int64_t)c * a.nchunk + k]);
  }
  __syncthreads();

  if (a.enable_spectrum) {
    // (hi, lo): the running sum of the groups' FP32 partial sums, exact
    // (two_sum); channels g, g + 32, ... in groups of 8, the group's loads
    // issued together
    float hi[4] = {0.f, 0.f, 0.f, 0.f}, lo[4] = {0.f, 0.f, 0.f, 0.f};
    float part[4] = {0.f, 0.f, 0.f, 0.f};
    for (int c0 = g; c0 < a.nchan; c0 += 32 * 8) {
      float v[8][4];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + 32 * u;
        if (c < a.nchan) {
          if (!in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status))
            v[u][0] = v[u][1] = v[u][2] = v[u][3] = 0.f;
          else if (valid == 4)
            raw_quad_values<DT>(ld_raw_quad<DT>(a.x, (int64_t)c * a.pitch + tq, keep), v[u]);
          else
            load_quad<DT>(a.x, (int64_t)c * a.pitch + tq, valid, v[u]);
        }
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + 32 * u;
        if (c >= a.nchan) break;
        const float2 m = s_mu[c];
        if (!s_cf[c]) {
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r < valid) part[r] += (v[u][r] - m.x) - m.y;
        }
      }
      if (c0 + 32 * 7 < a.nchan) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          two_sum_acc(hi[r], lo[r], part[r]);
          part[r] = 0.f;
        }
      }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      two_sum_acc(hi[r], lo[r], part[r]);
      s_fh[g][4 * q + r] = hi[r];
      s_fl[g][4 * q + r] = lo[r];
    }
    __syncthreads();
    if (tid < 32) {
      bool flag = false;
      if (t0 + tid < a.nsamp) {
        float mh = 0.f, ml = 0.f;
        for (int w = 0; w < 32; ++w) {
          two_sum_acc(mh, ml, s_fh[w][tid]);
          ml += s_fl[w][tid];
        }
        flag = (double)mh + (double)ml > a.spec_thr[k];
      }
      const unsigned bits = __ballot_sync(0xffffffffu, flag);
      if (tid == 0) {
        s_word = bits;
        if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = bits;
        if (bits) atomicAdd(a.spec_nflag, __popc(bits));
      }
    }
  } else if (tid == 0) {
    s_word = 0u;
    if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = 0u;
  }
  __syncthreads();
  const unsigned word = s_word;
  bool sflag[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) sflag[r] = (word >> (4 * q + r)) & 1u;
  if (valid == 0) return;

  // pass 2: y = x - mu (flagged -> 0) in FP32, or the 16-bit stored samples
  // x~ (flagged -> b16), or x~ - b16 in FP32 (stage_f32); 8 channels' loads
  // issued together
  for (int c0 = g; c0 < a.nchan; c0 += 32 * 8) {
    uint4 raw[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + 32 * u;
      if (c < a.nchan && valid == 4 && in_bounds((int64_t)c * a.pitch + tq, 4, a.x_elems, a.status))
        raw[u] = ld_raw_quad<DT>(a.x, (int64_t)c * a.pitch + tq, drop);
      else
        raw[u] = make_uint4(0u, 0u, 0u, 0u);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + 32 * u;
      if (c >= a.nchan) break;
      if (!in_bounds((int64_t)c * ypitch + tq, valid, a.y_elems, a.status)) continue;
      const bool cfl = s_cf[c] != 0;
      bool fl[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) fl[r] = sflag[r] || cfl;
      if constexpr (kStagedF32<DT>) {
        float v[4];
        if (valid == 4)
          raw_quad_values<DT>(raw[u], v);
        else
          load_quad<DT>(a.x, (int64_t)c * a.pitch + tq, valid, v);
        const float2 m = s_mu[c];
        float o[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) o[r] = fl[r] ? 0.f : (v[r] - m.x) - m.y;
        store_staged_f32_hint(yv, ypitch, c, tq, o, valid, drop);
      } else {
        unsigned short h[4];
        if (valid == 4) {
          h[0] = raw[u].x & 0xffff, h[1] = raw[u].x >> 16, h[2] = raw[u].y & 0xffff, h[3] = raw[u].y >> 16;
        } else {
          const unsigned short* src = static_cast<const unsigned short*>(a.x) + (int64_t)c * a.pitch + tq;
#pragma unroll
          for (int r = 0; r < 4; ++r) h[r] = r < valid ? __ldg(src + r) : 0;
        }
        const unsigned short b = s_b16[c];
#pragma unroll
        for (int r = 0; r < 4; ++r) h[r] = fl[r] ? b : h[r];
        if (a.stage_f32) {
          // y = x~ - b, one rounding of the difference of two exactly
          // converted stored values; flagged samples give exactly 0
          const float bf = bits_to_float<DT>(b);
          const float o[4] = {bits_to_float<DT>(h[0]) - bf, bits_to_float<DT>(h[1]) - bf,
                              bits_to_float<DT>(h[2]) - bf, bits_to_float<DT>(h[3]) - bf};
          store_staged_f32_hint(yv, ypitch, c, tq, o, valid, drop);
        } else {
          unsigned short* dst = static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq;
          if (valid == 4) {
            st_hint8(dst, make_uint2((unsigned)h[0] | ((unsigned)h[1] << 16), (unsigned)h[2] | ((unsigned)h[3] << 16)),
                     drop);
          } else {
            for (int r = 0; r < valid; ++r) dst[r] = h[r];
          }
        }
      }
    }
  }
}

// A3 + A4 for 8-bit data under the same conditions (W a multiple of 32,
// channels' parameters in shared memory): the exact integer spectrum sums of
// spectrum_substitute_kernel (sum of x over the unflagged channels against
// the sum of their offsets: N S_c with block statistics, b_c otherwise), then
// x~ (flagged -> b_c) widened to 16-bit integers; eight channels' 4-byte loads
// in flight per thread.
__global__ void __launch_bounds__(kThreads) spectrum_substitute_tile_u8(RfiArgs a, void* __restrict__ yv,
                                                                        int64_t ypitch) {
  extern __shared__ __align__(16) unsigned char s_dyn[];
  long long* s_off = reinterpret_cast<long long*>(s_dyn);          // [nchan] S_c or b_c
  int* s_b = reinterpret_cast<int*>(s_off + a.nchan);              // [nchan] b_c
  uint8_t* s_cf = reinterpret_cast<uint8_t*>(s_b + a.nchan);       // [nchan] chunk flag
  __shared__ long long s_i[32][33];
  __shared__ unsigned s_word;
  const int tid = threadIdx.x;
  const int g = tid >> 3, q = tid & 7;
  const int64_t t0 = (int64_t)blockIdx.x * 32;
  const int64_t tq = t0 + 4 * q;
  const int64_t left = a.nsamp - tq;
  const int valid = left >= 4 ? 4 : (left > 0 ? (int)left : 0);
  const int k = (int)(t0 / a.W);
  const bool ext = a.stats_mode == TP_STATS_EXTERNAL || a.fit || a.run;
  for (int c = tid; c < a.nchan; c += kThreads) {
    s_b[c] = a.bint[c];
    s_off[c] = ext ? (long long)a.bint[c] : a.S[c];
    s_cf[c] = (uint8_t)(a.chan_nflag[c] != 0 && a.chunk_flag[(int64_t)c * a.nchunk + k]);
  }
  __syncthreads();
  const unsigned char* xb = static_cast<const unsigned char*>(a.x);
  // the 4 samples of channel c at tq (those past the window read as 0)
  auto load4 = [&](int c) -> unsigned {
    if (valid == 4) return __ldg(reinterpret_cast<const unsigned*>(xb + (int64_t)c * a.pitch + tq));
    unsigned w = 0u;
    for (int r = 0; r < valid; ++r) w |= (unsigned)__ldg(xb + (int64_t)c * a.pitch + tq + r) << (8 * r);
    return w;
  };

  if (a.enable_spectrum) {
    // the thread's four samples summed as packed 16-bit lanes (samples 0, 2 in
    // plo, 1, 3 in phi): a lane takes at most kTileMaxChannels / 32 = 128
    // values below 256, so none carries into the next; samples past the
    // window load as 0.  The offsets of an unflagged channel are the same for
    // the four samples: summed once per channel.
    unsigned plo = 0u, phi = 0u;
    long long so = 0;
    for (int c0 = g; c0 < a.nchan; c0 += 32 * 8) {
      unsigned w[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + 32 * u;
        w[u] = c < a.nchan && in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status) ? load4(c) : 0u;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + 32 * u;
        if (c >= a.nchan) break;
        if (s_cf[c]) continue;
        plo += w[u] & 0x00ff00ffu;
        phi += (w[u] >> 8) & 0x00ff00ffu;
        so += s_off[c];
      }
    }
    const int sx[4] = {(int)(plo & 0xffffu), (int)(phi & 0xffffu), (int)(plo >> 16), (int)(phi >> 16)};
    long long sS[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) sS[r] = r < valid ? so : 0;
    const long long N = a.nsamp;
#pragma unroll
    for (int r = 0; r < 4; ++r) s_i[g][4 * q + r] = ext ? (long long)sx[r] - sS[r] : N * (long long)sx[r] - sS[r];
    __syncthreads();
    if (tid < 32) {
      bool flag = false;
      if (t0 + tid < a.nsamp) {
        long long m = 0;
        for (int w = 0; w < 32; ++w) m += s_i[w][tid];
        flag = (double)m > a.spec_thr[k];
      }
      const unsigned bits = __ballot_sync(0xffffffffu, flag);
      if (tid == 0) {
        s_word = bits;
        if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = bits;
        if (bits) atomicAdd(a.spec_nflag, __popc(bits));
      }
    }
  } else if (tid == 0) {
    s_word = 0u;
    if (t0 < a.nsamp) a.spec_bits[t0 >> 5] = 0u;
  }
  __syncthreads();
  const unsigned word = s_word;
  bool sflag[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) sflag[r] = (word >> (4 * q + r)) & 1u;
  const bool sany = ((word >> (4 * q)) & 0xfu) != 0u;
  if (valid == 0) return;
  const uint64_t drop = l2_policy(false);
  for (int c0 = g; c0 < a.nchan; c0 += 32 * 8) {
    unsigned w[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + 32 * u;
      w[u] = c < a.nchan && in_bounds((int64_t)c * a.pitch + tq, valid, a.x_elems, a.status) ? load4(c) : 0u;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + 32 * u;
      if (c >= a.nchan) break;
      if (!in_bounds((int64_t)c * ypitch + tq, valid, a.y_elems, a.status)) continue;
      const bool cfl = s_cf[c] != 0;
      const unsigned b = (unsigned)s_b[c];
      unsigned short* dst = static_cast<unsigned short*>(yv) + (int64_t)c * ypitch + tq;
      if (valid == 4 && !cfl && !sany) {
        // no sample of the quad is flagged: widen the four bytes to 16-bit
        // lanes with two byte permutes
        st_hint8(dst, make_uint2(__byte_perm(w[u], 0u, 0x4140), __byte_perm(w[u], 0u, 0x4342)), drop);
        continue;
      }
      unsigned h[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) h[r] = (sflag[r] || cfl) ? b : ((w[u] >> (8 * r)) & 0xffu);
      if (valid == 4) {
        st_hint8(dst, make_uint2(h[0] | (h[1] << 16), h[2] | (h[3] << 16)), drop);
      } else {
        for (int r = 0; r < valid; ++r) dst[r] = (unsigned short)h[r];
      }
    }
  }
}

// ---- fitted bandpass (Sec. 2.2.1 "Bandpass Correction") ---------------------------
//
// bandpass_fit_kernel (one CTA): local excess of each block mean over its
// neighbours' mean, e_c = mu_c - (mu_{c-1} + mu_{c+1}) / 2 (one neighbour at
// the band edges); channels with e_c > tau_mask * 1.4826 * median |e| (the
// lower middle of the sorted values, from a bitonic sort in shared memory)
// are masked and take the mean of their nearest unmasked neighbours; the
// result is fitted by least squares with Legendre polynomials P_0 .. P_p of
// x_c = (2c - (N - 1)) / (N - 1) (normal equations in binary64, Gaussian
// elimination with partial pivoting); b_c and the RMSE of the fit go to the
// beam, and b_c replaces the block mean as the value the spectrum and staging
// stages subtract (8-bit data: floor(b_c + 1/2); 16-bit data: b_c in the
// storage format).
constexpr int kFitThreads = 1024;

__global__ void __launch_bounds__(kFitThreads) bandpass_fit_kernel(RfiArgs a) {
  extern __shared__ double s_sort[];  // next power of two >= nchan
  const int N = a.nchan;
  int P = 1;
  while (P < N) P <<= 1;
  const double* mu = a.mu;
  double* e = a.fit_work;
  double* mi = a.fit_work + N;
  for (int c = threadIdx.x; c < P; c += kFitThreads) {
    double v = INFINITY;
    if (c < N) {
      double x;
      if (N == 1) x = 0.0;
      else if (c == 0) x = __dsub_rn(mu[0], mu[1]);
      else if (c == N - 1) x = __dsub_rn(mu[N - 1], mu[N - 2]);
      else x = __dsub_rn(mu[c], __ddiv_rn(__dadd_rn(mu[c - 1], mu[c + 1]), 2.0));
      e[c] = x;
      v = fabs(x);
    }
    s_sort[c] = v;
  }
  __syncthreads();
  // bitonic sort of s_sort[0 .. P), ascending
  for (int k = 2; k <= P; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < P; i += kFitThreads) {
        const int l = i ^ j;
        if (l > i) {
          const double x = s_sort[i], y = s_sort[l];
          const bool up = (i & k) == 0;
          if ((x > y) == up) s_sort[i] = y, s_sort[l] = x;
        }
      }
      __syncthreads();
    }
  __shared__ double s_thr;
  __shared__ int s_nmask;
  if (threadIdx.x == 0) {
    s_thr = __dmul_rn(a.tau_mask, __dmul_rn(1.4826, s_sort[(N - 1) / 2]));
    s_nmask = 0;
  }
  __syncthreads();
  const double thr = s_thr;
  int nm = 0;
  for (int c = threadIdx.x; c < N; c += kFitThreads) nm += e[c] > thr ? 1 : 0;
  atomicAdd(&s_nmask, nm);
  __syncthreads();
  const bool none = s_nmask == N;  // every channel masked: mask none
  for (int c = threadIdx.x; c < N; c += kFitThreads) a.fit_masked[c] = (uint8_t)(!none && e[c] > thr);
  __syncthreads();
  // interpolation of masked channels from their nearest unmasked neighbours
  for (int c = threadIdx.x; c < N; c += kFitThreads) {
    double v = mu[c];
    if (a.fit_masked[c]) {
      int l = c - 1, r = c + 1;
      while (l >= 0 && a.fit_masked[l]) --l;
      while (r < N && a.fit_masked[r]) ++r;
      if (l >= 0 && r < N) v = __ddiv_rn(__dadd_rn(mu[l], mu[r]), 2.0);
      else if (l >= 0) v = mu[l];
      else if (r < N) v = mu[r];
    }
    mi[c] = v;
  }
  __syncthreads();
  // normal equations: G[j][k] = sum_c P_j P_k (k <= j), r[j] = sum_c P_j mi_c
  const int p = a.fit_order, np1 = p + 1;
  constexpr int kG = (kMaxFitOrder + 1) * (kMaxFitOrder + 2) / 2;
  double g[kG + kMaxFitOrder + 1];
#pragma unroll
  for (int i = 0; i < kG + kMaxFitOrder + 1; ++i) g[i] = 0.0;
  const double half = N > 1 ? (double)(N - 1) : 1.0;
  for (int c = threadIdx.x; c < N; c += kFitThreads) {
    double L[kMaxFitOrder + 1];
    const double x = N > 1 ? __ddiv_rn((double)(2 * c - (N - 1)), half) : 0.0;
    L[0] = 1.0;
    if (p >= 1) L[1] = x;
    for (int i = 2; i <= p; ++i)
      L[i] = __ddiv_rn(__dsub_rn(__dmul_rn(__dmul_rn(L[i - 1], x), (double)(2 * i - 1)),
                                 __dmul_rn(L[i - 2], (double)(i - 1))),
                       (double)i);
    int q = 0;
    for (int j = 0; j < np1; ++j)
      for (int k = 0; k <= j; ++k) g[q++] += L[j] * L[k];
    for (int j = 0; j < np1; ++j) g[kG + j] += L[j] * mi[c];
  }
  __shared__ double s_g[kFitThreads / 32][kG + kMaxFitOrder + 1];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = 0; i < kG + kMaxFitOrder + 1; ++i) {
    double v = g[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) s_g[warp][i] = v;
  }
  __syncthreads();
  __shared__ double s_coef[kMaxFitOrder + 1];
  if (threadIdx.x == 0) {
    double A[kMaxFitOrder + 1][kMaxFitOrder + 2];
    for (int j = 0, q = 0; j < np1; ++j)
      for (int k = 0; k <= j; ++k, ++q) {
        double v = 0.0;
        for (int w = 0; w < kFitThreads / 32; ++w) v += s_g[w][q];
        A[j][k] = v;
        A[k][j] = v;
      }
    for (int j = 0; j < np1; ++j) {
      double v = 0.0;
      for (int w = 0; w < kFitThreads / 32; ++w) v += s_g[w][kG + j];
      A[j][np1] = v;
    }
    // Gaussian elimination with partial pivoting
    for (int col = 0; col < np1; ++col) {
      int piv = col;
      for (int r = col + 1; r < np1; ++r)
        if (fabs(A[r][col]) > fabs(A[piv][col])) piv = r;
      if (piv != col)
        for (int k = 0; k <= np1; ++k) {
          const double t = A[col][k];
          A[col][k] = A[piv][k];
          A[piv][k] = t;
        }
      const double d = A[col][col];
      for (int r = col + 1; r < np1; ++r) {
        const double f = d != 0.0 ? A[r][col] / d : 0.0;
        for (int k = col; k <= np1; ++k) A[r][k] -= f * A[col][k];
      }
    }
    for (int j = np1 - 1; j >= 0; --j) {
      double v = A[j][np1];
      for (int k = j + 1; k < np1; ++k) v -= A[j][k] * s_coef[k];
      s_coef[j] = A[j][j] != 0.0 ? v / A[j][j] : 0.0;
    }
  }
  __syncthreads();
  // fitted values, RMSE, and the values the later stages subtract
  double ss = 0.0;
  for (int c = threadIdx.x; c < N; c += kFitThreads) {
    double L[kMaxFitOrder + 1];
    const double x = N > 1 ? __ddiv_rn((double)(2 * c - (N - 1)), half) : 0.0;
    L[0] = 1.0;
    if (p >= 1) L[1] = x;
    for (int i = 2; i <= p; ++i)
      L[i] = __ddiv_rn(__dsub_rn(__dmul_rn(__dmul_rn(L[i - 1], x), (double)(2 * i - 1)),
                                 __dmul_rn(L[i - 2], (double)(i - 1))),
                       (double)i);
    double b = 0.0;
    for (int j = 0; j < np1; ++j) b += s_coef[j] * L[j];
    a.bfit[c] = b;
    const double r = b - mi[c];
    ss += r * r;
    const float hi = (float)b;
    a.mu_hi[c] = hi;
    a.mu_lo[c] = (float)(b - (double)hi);
    if (a.dtype == TP_U8) a.bint[c] = (int)floor(__dadd_rn(b, 0.5));
    if (a.dtype == TP_F16 || a.dtype == TP_BF16) a.b16[c] = storage_bits(a.dtype, b);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  __shared__ double s_ss[kFitThreads / 32];
  if (lane == 0) s_ss[warp] = ss;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < kFitThreads / 32; ++w) t += s_ss[w];
    *a.rmse = __dsqrt_rn(__ddiv_rn(t, (double)N));
  }
}

// Chunk test against the fitted bandpass (one CTA per channel): chunk k
// exceeds when sum(x - b_c) > tau_c * rmse * n_k (float chunk sums are
// relative to the channel's pivot; 8-bit ones are exact integers).
__global__ void __launch_bounds__(kThreads) fit_chunk_test_kernel(RfiArgs a, const void* chunk_sums) {
  const int c = blockIdx.x;
  const double b = a.bfit[c];
  const double tr = __dmul_rn(a.tau_c, *a.rmse);
  const bool single = a.W <= 256;
  for (int k = threadIdx.x; k < a.nchunk; k += kThreads) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t n = (lo + a.W < a.nsamp ? lo + a.W : a.nsamp) - lo;
    const int64_t idx = (int64_t)c * a.nchunk + k;
    double ex;
    if (a.dtype == TP_U8) {
      ex = __dsub_rn((double)static_cast<const longlong2*>(chunk_sums)[idx].x, __dmul_rn((double)n, b));
    } else {
      const double cs = single ? (double)static_cast<const float2*>(chunk_sums)[idx].x
                               : static_cast<const double2*>(chunk_sums)[idx].x;
      ex = __dsub_rn(cs, __dmul_rn((double)n, __dsub_rn(b, (double)a.pivot[c])));
    }
    a.chunk_raw[idx] = (uint8_t)(ex > __dmul_rn(tr, (double)n));
  }
}

// Running statistics (reading R15), one thread per channel: the block's own
// mean and variance folded into the previous state with weight alpha,
//   mu_run = alpha mu + (1 - alpha) mu_prev, var_run = alpha sigma^2 + (1 - alpha) var_prev
// (binary64, in this order; the stream's first block starts the state), and
// the block's statistics replaced by the running ones in every form the later
// stages read (mu, sigma, the split FP32 mean, the integer and 16-bit
// bandpass values).
__global__ void __launch_bounds__(kThreads) running_update_kernel(RfiArgs a) {
  const int c = blockIdx.x * kThreads + threadIdx.x;
  if (c >= a.nchan) return;
  double mu = a.mu[c];
  double var = __dmul_rn(a.sigma[c], a.sigma[c]);
  if (!a.run_first) {
    const double w = __dsub_rn(1.0, a.run_alpha);
    mu = __dadd_rn(__dmul_rn(a.run_alpha, mu), __dmul_rn(w, a.run_prev_mu[c]));
    var = __dadd_rn(__dmul_rn(a.run_alpha, var), __dmul_rn(w, a.run_prev_var[c]));
  }
  a.run_mu[c] = mu;
  a.run_var[c] = var;
  a.mu[c] = mu;
  a.sigma[c] = __dsqrt_rn(var);
  const float hi = (float)mu;
  a.mu_hi[c] = hi;
  a.mu_lo[c] = (float)(mu - (double)hi);
  a.bint[c] = (int)floor(__dadd_rn(mu, 0.5));
  if (a.dtype == TP_F16 || a.dtype == TP_BF16) a.b16[c] = storage_bits(a.dtype, mu);
}

// Channel test with running statistics (R5 with the running mean and spread):
// chunk k of channel c exceeds when sum(x - mu_run) > tau_c sigma_run
// sqrt(n_k); float chunk sums are relative to the channel's pivot, 8-bit ones
// exact integers (there the bandpass value floor(mu_run + 1/2) is subtracted,
// as for external statistics).
__global__ void __launch_bounds__(kThreads) running_chunk_test_kernel(RfiArgs a, const void* chunk_sums) {
  const int c = blockIdx.x;
  const double tsig = __dmul_rn(a.tau_c, a.sigma[c]);
  const bool single = a.W <= 256;
  for (int k = threadIdx.x; k < a.nchunk; k += kThreads) {
    const int64_t lo = (int64_t)k * a.W;
    const int64_t n = (lo + a.W < a.nsamp ? lo + a.W : a.nsamp) - lo;
    const int64_t idx = (int64_t)c * a.nchunk + k;
    double ex;
    if (a.dtype == TP_U8) {
      ex = (double)(static_cast<const longlong2*>(chunk_sums)[idx].x - n * (long long)a.bint[c]);
    } else {
      const double cs = single ? (double)static_cast<const float2*>(chunk_sums)[idx].x
                               : static_cast<const double2*>(chunk_sums)[idx].x;
      ex = __dsub_rn(cs, __dmul_rn((double)n, __dsub_rn(a.mu[c], (double)a.pivot[c])));
    }
    a.chunk_raw[idx] = (uint8_t)(ex > __dmul_rn(tsig, __dsqrt_rn((double)n)));
  }
}

// Pitched row copy in 16-byte units: CTA (x, y) copies kThreads kCopyUnroll
// consecutive units of rows y, y + gridDim.y, ...; all loads of a thread are
// issued before its stores.
constexpr int kCopyUnroll = 4;

__global__ void __launch_bounds__(kThreads) copy_rows_kernel(int4* __restrict__ dst, int64_t dpitch,
                                                             const int4* __restrict__ src, int64_t spitch,
                                                             int64_t row_units, int nrows) {
  constexpr int64_t span = (int64_t)kThreads * kCopyUnroll;
  for (int r = blockIdx.y; r < nrows; r += gridDim.y) {
    const int4* s = src + (int64_t)r * spitch;
    int4* d = dst + (int64_t)r * dpitch;
    for (int64_t base = (int64_t)blockIdx.x * span + threadIdx.x; base < row_units; base += (int64_t)gridDim.x * span) {
      int4 v[kCopyUnroll];
#pragma unroll
      for (int u = 0; u < kCopyUnroll; ++u) {
        const int64_t i = base + (int64_t)u * kThreads;
        if (i < row_units) v[u] = __ldcs(s + i);
      }
#pragma unroll
      for (int u = 0; u < kCopyUnroll; ++u) {
        const int64_t i = base + (int64_t)u * kThreads;
        if (i < row_units) d[i] = v[u];
      }
    }
  }
}

}  // namespace

cudaError_t copy_rows(void* dst, size_t dpitch, const void* src, size_t spitch, size_t row_bytes, int nrows,
                      cudaStream_t s, int* kernels) {
  if (nrows <= 0 || row_bytes == 0) return cudaSuccess;
  const bool vec = ((uintptr_t)dst | (uintptr_t)src | dpitch | spitch | row_bytes) % 16 == 0;
  if (!vec) return cudaMemcpy2DAsync(dst, dpitch, src, spitch, row_bytes, nrows, cudaMemcpyDeviceToDevice, s);
  const int64_t units = (int64_t)(row_bytes / 16);
  const int64_t span = (int64_t)kThreads * kCopyUnroll;
  const int64_t gx = (units + span - 1) / span;
  const dim3 grid((unsigned)(gx < 1024 ? gx : 1024), (unsigned)(nrows < 65535 ? nrows : 65535));
  copy_rows_kernel<<<grid, kThreads, 0, s>>>(static_cast<int4*>(dst), (int64_t)(dpitch / 16),
                                             static_cast<const int4*>(src), (int64_t)(spitch / 16), units, nrows);
  if (kernels) ++*kernels;
  return cudaGetLastError();
}

template <int DT>
cudaError_t launch_tile(const RfiArgs& a, void* y, int64_t ypitch, unsigned blocks, size_t sm, cudaStream_t s) {
  if (sm > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(spectrum_substitute_tile<DT>,
                                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  spectrum_substitute_tile<DT><<<blocks, kThreads, sm, s>>>(a, y, ypitch);
  return cudaGetLastError();
}

cudaError_t launch_rfi(const RfiArgs& a, void* chunk_sums, void* y, int64_t ypitch, cudaStream_t s, int* kernels) {
  int nk = 2;  // the statistics kernels
  cudaError_t e = launch_stats(a, chunk_sums, s);
  if (e != cudaSuccess) return e;
  const int64_t nflag_bytes = (int64_t)a.nchan * a.nchunk;
  if (a.fit) {
    int P = 1;
    while (P < a.nchan) P <<= 1;
    const size_t sm = sizeof(double) * (size_t)P;
    e = cudaFuncSetAttribute(bandpass_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    bandpass_fit_kernel<<<1, kFitThreads, sm, s>>>(a);
    ++nk;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.enable_channel) {
      fit_chunk_test_kernel<<<a.nchan, kThreads, 0, s>>>(a, chunk_sums);
      ++nk;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  if (a.run) {
    running_update_kernel<<<(a.nchan + kThreads - 1) / kThreads, kThreads, 0, s>>>(a);
    ++nk;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (a.enable_channel) {
      running_chunk_test_kernel<<<a.nchan, kThreads, 0, s>>>(a, chunk_sums);
      ++nk;
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  if (a.enable_channel) {
    dilate_kernel<<<(a.nchan + kWarps - 1) / kWarps, kThreads, 0, s>>>(a);
    ++nk;
  } else {
    e = cudaMemsetAsync(a.chunk_raw, 0, nflag_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.chunk_flag, 0, nflag_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(a.chan_nflag, 0, sizeof(int) * a.nchan, s);
  }
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  nk += 2;  // spectrum thresholds and substitution
  if (kernels) *kernels += nk;
  spectrum_threshold_kernel<<<(unsigned)((a.nchunk + kWarps - 1) / kWarps), kThreads, 0, s>>>(a);
  const unsigned blocks = (unsigned)((a.nsamp + 31) / 32);
  if (a.dtype == TP_U8 && a.W % 32 == 0 && a.nchan <= kTileMaxChannels) {
    const size_t sm = (size_t)a.nchan * (sizeof(long long) + sizeof(int) + 1);
    if (sm > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(spectrum_substitute_tile_u8,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
    }
    spectrum_substitute_tile_u8<<<blocks, kThreads, sm, s>>>(a, y, ypitch);
    return cudaGetLastError();
  }
  if (a.dtype != TP_U8 && a.W % 32 == 0 && a.nchan <= kTileMaxChannels) {
    const size_t sm = (size_t)a.nchan * (sizeof(float2) + sizeof(unsigned short) + 1);
    if (a.dtype == TP_C16) return launch_tile<TP_C16>(a, y, ypitch, blocks, sm, s);
    if (a.dtype == TP_F16) return launch_tile<TP_F16>(a, y, ypitch, blocks, sm, s);
    if (a.dtype == TP_BF16) return launch_tile<TP_BF16>(a, y, ypitch, blocks, sm, s);
    return launch_tile<TP_F32>(a, y, ypitch, blocks, sm, s);
  }
  if (a.dtype == TP_C16)
    spectrum_substitute_kernel<TP_C16><<<blocks, kThreads, 0, s>>>(a, y, ypitch);
  else if (a.dtype == TP_U8)
    spectrum_substitute_kernel<TP_U8><<<blocks, kThreads, 0, s>>>(a, y, ypitch);
  else if (a.dtype == TP_F16)
    spectrum_substitute_kernel<TP_F16><<<blocks, kThreads, 0, s>>>(a, y, ypitch);
  else if (a.dtype == TP_BF16)
    spectrum_substitute_kernel<TP_BF16><<<blocks, kThreads, 0, s>>>(a, y, ypitch);
  else
    spectrum_substitute_kernel<TP_F32><<<blocks, kThreads, 0, s>>>(a, y, ypitch);
  return cudaGetLastError();
}

// A1-A2 alone (bandpass statistics, channel exceedances and their dilation)
// with the chunk sums in caller-chosen scratch; used by the entry point that
// allocates nothing.
cudaError_t launch_channel_stats(const RfiArgs& a, void* chunk_sums, cudaStream_t s) {
  cudaError_t e = launch_stats(a, chunk_sums, s);
  if (e != cudaSuccess) return e;
  const int64_t nflag_bytes = (int64_t)a.nchan * a.nchunk;
  if (a.enable_channel) {
    dilate_kernel<<<(a.nchan + kWarps - 1) / kWarps, kThreads, 0, s>>>(a);
    return cudaGetLastError();
  }
  e = cudaMemsetAsync(a.chunk_raw, 0, nflag_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.chunk_flag, 0, nflag_bytes, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(a.chan_nflag, 0, sizeof(int) * a.nchan, s);
  return e;
}

}  // namespace tp
